"""Benchmark of the V-FPI hot path on GB300.

Workload: the 128x128x32 mass-spring lattice draped on a sinusoid+noise
heightfield (1,572,864 DOF, 13,716,856 3x3 blocks, 16,384 contacts with
mu ~ U[0.2, 0.8]), FP32 with FP64 residual reduction and position update.  One
step = one time step of the solver: reset the warm start, run Alg. 1 to
theta < theta_th or l = l_max (200) on the device, integrate x += h v_hat in
FP64.  ``value`` is DOF x sweeps / device time (DOF-iterations per second).

``--impl reference`` times the FP64 CPU oracle on the same workload instead
(a bounded number of sweeps per step).  Under torchrun each rank runs an
independent replica (``value``, weak scaling); the same scene is then also
split into one z-slab per rank and solved with a halo exchange per sweep over
NCCL (key ``sharded``, strong scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import resource
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "V-FPI DOF-iters/s & % HBM roofline; batched env-steps/s; adjoint/forward ratio"
UNIT = "DOF-iter/s"
WORKLOAD = "terrain_lattice_128x128x32"
THETA_TH = 1e-6          # RMS residual threshold (m/s per DOF)
L_MAX = 200
FALLBACK_HBM_GBS = 6800.0

BATCH_CHEBYSHEV = (5, 1.0)   # Alg. 3 for the batched env steps' second figure
ADJ_THETA_REL = 1e-4        # adjoint stop: ||u^{l+1} - u^l|| < 1e-4 ||dL/dv|| (rms, per scene)
ADJ_L_MAX = 5000
ADJ_CHEBYSHEV = (5, 1.0)    # Alg. 3 on the adjoint iteration (slow start, under-relaxation)
# ncu DRAM traffic (read + write bytes per sweep) of the single-scene solve
# kernel, keyed by (hash of the CUDA sources it was captured from, kernel
# variant), each captured at the variant's default CTA count; stale entries
# read as null (the grid kernel's ncu summary gives the captures)
NCU_TRAFFIC = {("0d1008fea7fe258c", 0): 554637560, ("0d1008fea7fe258c", 7): 553524952,
               ("0d1008fea7fe258c", 28): 388417174, ("0d1008fea7fe258c", 29): 387921396}
# the same for the batched kernel: (DRAM read + write bytes, algorithmic bytes)
# of one captured env-step solve launch (the bench's launch log gives the
# captured launch's own count), keyed by (source hash, storage of A as
# Solver.storage() names it, threads per CTA)
NCU_BATCH_TRAFFIC = {("0d1008fea7fe258c", "blocks6", 256): (114027696568, 172972435132)}
# kernel-name notes for the compressed storages of A (the fraction keeps the
# 40-byte full-BSR count per block, so on these it is an effective one)
STORAGE_NOTE = {
    "symmetric": " (symmetric storage; effective fraction)",
    "blocks6": " on symmetric blocks (6 values per block streamed; effective fraction)",
}


def source_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2201_09212_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def algorithmic_bytes_per_sweep(sc, esz=4) -> int:
    """Bytes one sweep must move at minimum with A as given (full BSR): every
    block and column index once, the row pointers, v^l read, b read, v^{l+1}
    written, W read, the contact records (R, mu, phi, node ids: 48 B) and
    lambda written (12 B)."""
    N, n, nnzb, n_c = sc.n_nodes, sc.n, sc.nnzb, sc.n_c
    vec = 4 * (N + 1) + 3 * esz * n + esz * N + n_c * (48 + 12)
    return nnzb * (9 * esz + 4) + vec


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(dist, device, elapsed_s: float, units: float):
    """Whole-job throughput over all ranks: the units every rank processed,
    summed, over the slowest rank's time (max over ranks).  Returns
    (units per second, max time, total units)."""
    if dist is None:
        return units / elapsed_s, elapsed_s, units
    import torch
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item()), float(u.item())


def cpu_oracle_rate(sc, sweeps: int):
    """Time the FP64 oracle's V-FPI sweeps on this host; returns
    (DOF-iter/s, effective cores, seconds)."""
    from oracle import vfpi as ov
    P = ov.make_problem(sc.row_ptr, sc.col_idx, sc.vals, sc.b, sc.node_i, sc.node_j, sc.R,
                        sc.mu, sc.phi)
    w = ov.frobenius_w(P)
    v = np.asarray(sc.v0, dtype=np.float64)
    ov.sweep(P, w, v)  # warm
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    for _ in range(sweeps):
        v = ov.sweep(P, w, v).v_next
    dt = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    return sc.n * sweeps / dt, max(1, round(cpu / dt)), dt


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def _oracle_block_worker(job, start, results):
    """One core's share of the all-core CPU baseline: the unmodified FP64
    oracle sweep (Alg. 1 + Alg. 2) on one z-slab of the scene -- its rows, and
    its halo as identity rows with b = 0 so that the block is a square problem
    -- timed over the same number of sweeps as the other workers, which start
    together."""
    from oracle import vfpi as ov
    P = ov.make_problem(*job["problem"])
    w = ov.frobenius_w(P)
    v = np.asarray(job["v0"], dtype=np.float64)
    ov.sweep(P, w, v)
    start.wait()
    t0 = time.perf_counter()
    for _ in range(job["sweeps"]):
        v = ov.sweep(P, w, v).v_next
    results.put(time.perf_counter() - t0)


def cpu_oracle_rate_all_cores(sc, dims, sweeps: int):
    """The FP64 oracle's sweep over all host cores: the scene split into one
    z-slab per core (the split of the multi-GPU path), every slab swept by the
    oracle in its own process, all at once; DOF-iterations per second over the
    slowest slab.  The halo exchange between sweeps is left out (the slabs'
    sweeps are timed back to back), so this bounds an all-core oracle from
    above.  Returns (rate, cores, seconds)."""
    import multiprocessing as mp
    from paper_2201_09212_gb300 import shard
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    cores = max(1, min(cores, sc.n_nodes // (dims[0] * dims[1])))
    ranges = shard.partition(sc.row_ptr, cores, align=dims[0] * dims[1])
    jobs = []
    for n0, n1 in ranges:
        halo = shard.halo_of(sc.row_ptr, sc.col_idx, n0, n1)
        r0, r1 = int(sc.row_ptr[n0]), int(sc.row_ptr[n1])
        cols = sc.col_idx[r0:r1].astype(np.int64)
        own = (cols >= n0) & (cols < n1)
        local = np.where(own, cols - n0, (n1 - n0) + np.searchsorted(halo, cols))
        nh = len(halo)
        row_ptr = np.concatenate([sc.row_ptr[n0:n1 + 1] - r0, (r1 - r0) + np.arange(1, nh + 1)])
        col_idx = np.concatenate([local, (n1 - n0) + np.arange(nh)])
        vals = np.concatenate([sc.vals[r0:r1].astype(np.float64), np.broadcast_to(np.eye(3), (nh, 3, 3))])
        b = np.concatenate([sc.b[3 * n0:3 * n1], np.zeros(3 * nh)])
        cm = (sc.node_i >= n0) & (sc.node_i < n1)
        v0 = np.concatenate([sc.v0[3 * n0:3 * n1], sc.v0.reshape(-1, 3)[halo].ravel()])
        jobs.append({"problem": (row_ptr, col_idx, vals, b, sc.node_i[cm] - n0, sc.node_j[cm],
                                 sc.R[cm], sc.mu[cm], sc.phi[cm]),
                     "v0": v0, "sweeps": sweeps})
    ctx = mp.get_context("spawn")   # this process already holds a CUDA context
    start, results = ctx.Barrier(len(jobs)), ctx.Queue()
    procs = [ctx.Process(target=_oracle_block_worker, args=(j, start, results)) for j in jobs]
    for p in procs:
        p.start()
    times = [results.get() for _ in procs]
    for p in procs:
        p.join()
    t = max(times)
    return sc.n * sweeps / t, len(jobs), t


def run_reference(args, sc):
    """The FP64 oracle as it stands on this host's cores: the problem and W
    are built once, then each step is one oracle V-FPI sweep over the whole
    workload (the bounded sample; about 0.15 s on one Grace core)."""
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    from oracle import vfpi as ov
    P = ov.make_problem(sc.row_ptr, sc.col_idx, sc.vals, sc.b, sc.node_i, sc.node_j, sc.R,
                        sc.mu, sc.phi)
    w = ov.frobenius_w(P)
    v = np.asarray(sc.v0, dtype=np.float64)
    per_step = 1
    for _ in range(args.warmup):
        v = ov.sweep(P, w, v).v_next
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(per_step):
            v = ov.sweep(P, w, v).v_next
    wall = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    cores = max(1, round(cpu / wall))
    value = sc.n * per_step * args.steps / wall
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "dof": sc.n, "blocks": sc.nnzb, "contacts": sc.n_c},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} FP64 oracle V-FPI sweep per step of the full workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batched_bench(args, torch, dev, stream, rank):
    """4,096 independent uneven lattices (192-5,184 DOF each) on the ground plane,
    one persistent CTA-per-scene launch per time step, the whole env step
    (dynamics harness: b = M v + h M g - kappa (A - M)(x - x0), phi = z / h; warm
    start; solve; x += h v_hat) captured in one CUDA graph.  Also times plain
    per-scene solves of a sample of scenes on the same GPU for comparison."""
    from paper_2201_09212_gb300 import scenes, vfpi
    sc = scenes.lattice_batch(args.batch_scenes, seed=scenes.SEED_BASE + 4 + 1000 * rank)
    meta = sc.meta
    S = len(meta["sides"])
    nq = meta["nodes"].astype(np.int64)
    dof_scene = np.repeat(np.arange(S), 3 * nq)
    comp = np.tile(np.arange(3), int(nq.sum()))
    h = sc.h
    g_dof = meta["gravity"][dof_scene, comp]
    kappa = (h * meta["k"] / meta["coef"])[dof_scene]
    T = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(dev)
    s = vfpi.Solver.from_scene(sc, theta_th=THETA_TH, l_max=L_MAX, norm="rms", stream=stream)
    s.set_velocity(torch.from_numpy(sc.v0).to(dev))
    from paper_2201_09212_gb300 import tune
    tuned = tune.tune(s, sweeps=20, reps=2)
    x0 = T(sc.x0, np.float64)
    x = x0.clone()
    v = T(sc.v0, np.float32)
    mass = T(sc.mass, np.float32)
    hg = T(h * sc.mass * g_dof, np.float32)
    kap = T(kappa, np.float32)
    zi = T(3 * sc.node_i.astype(np.int64) + 2, np.int64)
    Au = torch.empty_like(v)
    b = torch.empty_like(v)
    phi = torch.empty(sc.n_c, dtype=torch.float32, device=dev)

    def env_step():
        u = (x - x0).float()
        s.matvec(u, out=Au)
        torch.mul(mass, v, out=b)
        b.add_(hg)
        b.sub_(kap * (Au - mass * u))
        torch.div(x.index_select(0, zi).float(), h, out=phi)
        s.set_rhs(b, phi)
        s.set_velocity(v)
        s.solve_async()
        s.integrate(x)
        s.get_velocity(out=v)

    n_dof = 3 * nq
    nc_q = np.bincount(np.searchsorted(sc.scene_ptr, sc.node_i, side="right") - 1, minlength=S)
    bytes_scene = np.array([
        algorithmic_bytes_per_sweep(type("Q", (), dict(n_nodes=int(n), n=3 * int(n), nnzb=int(bq), n_c=int(c)))())
        for n, bq, c in zip(nq, np.diff(sc.row_ptr[sc.scene_ptr]), nc_q)])
    launch_log = []

    def log_launch(kind):
        # the solve launches in program order, each with its own algorithmic
        # byte count (per-scene sweeps x per-scene bytes), so that a profiler
        # capture of launch k can be set against its count
        it, _, _ = s.status()
        launch_log.append({"launch": len(launch_log), "kind": kind,
                           "scene_sweeps": int(it.sum()),
                           "alg_bytes": int((it * bytes_scene).sum())})

    def timed_steps(log=False):
        # from the initial state: warm-up steps, one graph per env step, timed replays
        x.copy_(x0)
        v.copy_(T(sc.v0, np.float32))
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                env_step()
                if log:
                    log_launch("warm-up")
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                env_step()
            for _ in range(2):
                g.replay()
                if log:
                    log_launch("replay before timing")
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            dof_iters, kms, its = 0, [], []
            t_total = 0.0
            for _ in range(args.batch_steps):
                ev0.record(stream)
                g.replay()
                ev1.record(stream)
                ev1.synchronize()
                t_total += ev0.elapsed_time(ev1) / 1e3
                it, _, _ = s.status()
                its.append(it.copy())
                dof_iters += int((n_dof * it).sum())
                kms.append(s.last_kernel_ms())
                if log and len(launch_log) < args.warmup + 5:
                    log_launch("timed")
        return t_total, np.array(its), dof_iters, kms

    t_total, its, dof_iters, kms = timed_steps(log=True)
    # the same env steps with Chebyshev acceleration (Alg. 3) of the solves:
    # the same stop test, reached in fewer sweeps
    s.set_chebyshev(*BATCH_CHEBYSHEV)
    t_cheb, its_cheb, _, _ = timed_steps()
    s.set_chebyshev(0)
    env_sps = S * args.batch_steps / t_total
    alg = float((its * bytes_scene[None, :]).sum(axis=1).mean())
    k_avg = float(np.mean(kms)) / 1e3
    # plain per-scene solves (one context per scene) on a sample, same tolerance
    rng = np.random.default_rng(0)
    sample = rng.choice(S, size=min(args.per_scene_sample, S), replace=False)
    per_ms = []
    for q in sample:
        n0, n1 = sc.scene_ptr[q], sc.scene_ptr[q + 1]
        r0, r1 = sc.row_ptr[n0], sc.row_ptr[n1]
        cm = (sc.node_i >= n0) & (sc.node_i < n1)
        with vfpi.Solver(sc.row_ptr[n0:n1 + 1] - r0, sc.col_idx[r0:r1] - n0, sc.vals[r0:r1],
                         sc.b[3 * n0:3 * n1], sc.node_i[cm] - n0, None, sc.R[cm], sc.mu[cm],
                         sc.phi[cm], theta_th=THETA_TH, l_max=L_MAX, norm="rms",
                         stream=stream) as s1:
            s1.set_velocity(sc.v0[3 * n0:3 * n1])
            for _ in range(2):
                s1.solve_async()
                s1.status()
            per_ms.append(s1.last_kernel_ms())
    per_scene_total = float(np.mean(per_ms)) / 1e3 * S
    first_batch = kms[0] / 1e3
    lay_b = s.layout()
    stor_b = s.storage()["storage"]
    threads = lay_b["threads"]
    var = int(tuned.get("kernel_variant", 0))
    kname = (f"k_solve_cluster<float,{threads}> (launch shape {var})" if 16 <= var <= 25
             else f"k_solve_scenes<float,{threads}>" + STORAGE_NOTE.get(stor_b, ""))
    tr_key = (source_hash(), stor_b, threads)
    tr_ratio = (NCU_BATCH_TRAFFIC[tr_key][0] / NCU_BATCH_TRAFFIC[tr_key][1]
                if tr_key in NCU_BATCH_TRAFFIC and (var < 16 or var == 30) else None)
    s.close()
    return {
        "workload": f"{S} lattices, side U{{4..12}}, {int(nq.sum()) * 3} DOF, {sc.nnzb} blocks, {sc.n_c} contacts",
        "env_steps_per_s": env_sps, "ms_per_env_step": 1e3 * t_total / args.batch_steps,
        "steps": args.batch_steps, "dof_iters_per_s": dof_iters / t_total,
        "iters_per_scene": {"mean": float(its.mean()), "min": int(its.min()), "max": int(its.max())},
        "solve_kernel": {"name": kname, "ms_avg": 1e3 * k_avg,
                         "achieved_gbs": alg / k_avg / 1e9, "frac": alg / k_avg / 1e9 / peaks()[0],
                         "traffic_over_algorithmic": tr_ratio,
                         # DRAM bytes actually moved (ncu ratio x algorithmic) over the live time
                         "dram_frac": (tr_ratio * alg / k_avg / 1e9 / peaks()[0]
                                       if tr_ratio else None)},
        "graph": "one CUDA graph per env step (harness, warm start, solve, integrate)",
        "layout": {"blocks": int(sc.nnzb), "stored_slots": int(lay_b["slots"]),
                   "padding": lay_b["slots"] / sc.nnzb - 1.0},
        "launch_log": launch_log,
        "with_chebyshev": {"l_s_u": list(BATCH_CHEBYSHEV),
                           "env_steps_per_s": S * args.batch_steps / t_cheb,
                           "ms_per_env_step": 1e3 * t_cheb / args.batch_steps,
                           "iters_per_scene": {"mean": float(its_cheb.mean()),
                                               "max": int(its_cheb.max())}},
        "per_scene_plain": {"sample": len(sample), "mean_solve_ms": float(np.mean(per_ms)),
                            "extrapolated_all_scenes_s": per_scene_total,
                            "batched_solve_s": first_batch,
                            "speedup": per_scene_total / first_batch},
    }


def sharded_bench(args, torch, dist, dev, sc, dims, rank, ws):
    """The single scene split into one z-slab per rank (a shard context per
    rank with its halo), Alg. 1 with the halo rows exchanged and the FP64
    residual summed over NCCL every sweep; whole-scene DOF-iterations per
    second over the slowest rank's time."""
    from paper_2201_09212_gb300 import shard
    ranges = shard.partition(sc.row_ptr, ws, align=dims[0] * dims[1])
    plan = shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, rank)
    comm = shard.TorchComm(dist, dev)
    v0 = torch.from_numpy(np.ascontiguousarray(sc.v0[3 * plan.n0:3 * plan.n1])).to(dev)
    kw = dict(n_dof=sc.n, theta_th=THETA_TH, l_max=L_MAX, norm="rms", device=dev)
    with shard.shard_solver(sc, plan) as eng:
        for _ in range(args.warmup):
            shard.solve(eng, plan, comm, v0, **kw)
        iters = []
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.sharded_steps):
            iters.append(shard.solve(eng, plan, comm, v0, **kw).iters)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
    _, t, _ = aggregate(dist, dev, t, 0.0)
    return {"workload": f"{WORKLOAD} in {ws} z-slabs", "ranges": ranges,
            "halo_nodes": int(len(plan.halo)), "steps": args.sharded_steps,
            "iters_per_step": float(np.mean(iters)), "ms_per_step": 1e3 * t / args.sharded_steps,
            "dof_iters_per_s": sc.n * float(np.sum(iters)) / t, "scaling": "strong",
            "note": "one launch and one host round trip per sweep (exchange, residual sum)"}


def sharded_one_gpu_bench(args, torch, dev, sc, dims, kernel_ms_per_sweep):
    """The host-driven loop of the split scene on one GPU: two z-slab shards
    in one process (shard.solve_local), Alg. 1 to the same stop test.  The
    shards' launches run one after the other, so the step time above the
    unsplit kernel's is the loop's own cost per sweep: two launches, the host
    round trip for the residual sum and the halo rows' exchange."""
    from paper_2201_09212_gb300 import shard
    ranges = shard.partition(sc.row_ptr, 2, align=dims[0] * dims[1])
    plans = [shard.make_plan(sc.row_ptr, sc.col_idx, sc.node_i, sc.node_j, ranges, r)
             for r in range(2)]
    engines = [shard.shard_solver(sc, pl) for pl in plans]
    v0 = torch.from_numpy(np.ascontiguousarray(sc.v0)).to(dev)
    kw = dict(n_dof=sc.n, theta_th=THETA_TH, l_max=L_MAX, norm="rms", device=dev)
    try:
        for _ in range(args.warmup):
            shard.solve_local(engines, plans, v0, **kw)
        iters = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.sharded_steps):
            iters.append(shard.solve_local(engines, plans, v0, **kw).iters)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
    finally:
        for e in engines:
            e.close()
    sweeps = float(np.sum(iters))
    return {"workload": f"{WORKLOAD} in 2 z-slabs, both on this GPU", "ranges": ranges,
            "halo_nodes": [int(len(pl.halo)) for pl in plans], "steps": args.sharded_steps,
            "iters_per_step": float(np.mean(iters)), "ms_per_step": 1e3 * t / args.sharded_steps,
            "dof_iters_per_s": sc.n * sweeps / t,
            "loop_us_per_sweep_over_unsplit_kernel": 1e6 * t / sweeps - 1e3 * kernel_ms_per_sweep,
            "note": "the shards' launches one after the other; no device exchange"}


def configs_bench(args, torch, dev, stream):
    """The other plain-V-FPI configurations, each solved from its initial
    state repeatedly (tuned launch shape; a 256 MB write between steps flushes
    L2): the 6x6x6 FP64 lattice and the 64x64x16 FEM block.  The FEM block's
    matrix (about 45 MB) fits in the 126 MB L2, so within a solve its sweeps
    run from L2 and the fraction of HBM is an effective one."""
    from paper_2201_09212_gb300 import scenes, tune, vfpi
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    out = {}
    for name, make, dtype, esz, theta, steps in (
            ("small_lattice_6x6x6_f64", lambda: scenes.small_lattice(np.float64), "f64", 8, 1e-9, 100),
            ("fem_block_64x64x16_f32", lambda: scenes.fem_block(), "f32", 4, 1e-6, 50)):
        sc = make()
        with vfpi.Solver.from_scene(sc, theta_th=theta, l_max=5000, norm="rms", dtype=dtype,
                                    stream=stream) as s:
            v0 = torch.from_numpy(sc.v0).to(dev)
            s.set_velocity(v0)
            # under the timing loop's condition (L2 flushed before each solve),
            # windows of 40 sweeps, best of 3
            tuned = tune.tune(s, sweeps=40, reps=3, condition="l2-flushed",
                              before_rep=lambda: flush.fill_(0.0))
            kms, its = [], []
            with torch.cuda.stream(stream):
                for k in range(3 + steps):
                    flush.fill_(float(k))
                    s.set_velocity(v0)
                    s.solve_async()
                    it, _, _ = s.status()
                    if k >= 3:
                        kms.append(s.last_kernel_ms())
                        its.append(int(it[0]))
            lay = s.layout()
        t = sum(kms) / 1e3
        bps = algorithmic_bytes_per_sweep(sc, esz)
        achieved = bps * sum(its) / t / 1e9
        out[name] = {"dof": sc.n, "blocks": sc.nnzb, "contacts": sc.n_c, "dtype": dtype,
                     "theta_th_rms": theta, "steps": steps, "iters_per_step": float(np.mean(its)),
                     "dof_iters_per_s": sc.n * sum(its) / t, "ms_per_solve": 1e3 * t / steps,
                     "achieved_gbs": achieved, "frac_of_hbm": achieved / peaks()[0],
                     "matrix_mb": sc.nnzb * (9 * esz + 4) / 1e6,
                     "path": "grid" if lay["path"] == 1 else "CTA-per-scene",
                     "launch": {k: tuned[k] for k in ("kernel_variant", "block_threads", "grid")},
                     "tuner_best": [[t["kernel_variant"], t["grid"], round(1e3 * t["ms_per_sweep"], 2)]
                                    for t in sorted(tuned.get("trials", []),
                                                    key=lambda t: t["ms_per_sweep"])[:5]],
                     "l2": "flushed between steps (256 MB write)"}
    return out


def adjoint_bench(args, torch, dev, stream):
    """256 rest-linearised 16x16x8 lattices (6,144 DOF each), a 64-step rollout
    differentiated by torch autograd through the adjoint kernel, checkpointed
    every 8 steps: wall time of the backward pass (recompute + adjoint solves)
    over the forward pass.  The adjoint solves stop relative to their load
    (dL/dv has the loss's scale) and use Alg. 3; a directional central
    difference of the loss checks the gradient."""
    from paper_2201_09212_gb300 import scenes, vfpi
    from paper_2201_09212_gb300.autograd import LatticeHarness, rollout
    sc = scenes.lattice_batch(args.adj_scenes, seed=scenes.SEED_BASE + 5, dims=(16, 16, 8))
    s = vfpi.Solver.from_scene(sc, theta_th=THETA_TH, l_max=L_MAX, norm="rms", stream=stream)
    # the adjoint's load dL/dv has the loss's scale: stop relative to it, and
    # accelerate the (linear) adjoint iteration with Alg. 3
    s.set_adjoint_tolerance(ADJ_THETA_REL, ADJ_L_MAX, relative=True)
    s.set_adjoint_chebyshev(*ADJ_CHEBYSHEV)
    s.set_velocity(torch.from_numpy(sc.v0).to(dev))
    from paper_2201_09212_gb300 import tune
    tuned = tune.tune(s, sweeps=20, reps=2)
    H = LatticeHarness(sc, dev)
    res = {}
    with torch.cuda.stream(stream):
        for rep in range(2):                       # first pass warms up
            v0 = torch.from_numpy(sc.v0).to(dev).requires_grad_(True)
            mu = torch.from_numpy(sc.mu).to(dev).requires_grad_(True)
            steps = 8 if rep == 0 else args.adj_steps
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x, _ = rollout(s, H, H.x_rest.clone(), v0, mu, steps, checkpoint=8)
            L = H.com_z(x).sum()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            L.backward()
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            res = {"forward_s": t1 - t0, "backward_s": t2 - t1,
                   "grad_norm_v0": float(v0.grad.norm()), "grad_norm_mu": float(mu.grad.norm())}
        # central differences of the loss along sign(grad) (g . d = ||g||_1: a
        # signal well above the forward's stop-test noise in the loss) for v0 and mu
        checks = {}
        for name, base, grad in (("v0", sc.v0, v0.grad), ("mu", sc.mu, mu.grad)):
            d = torch.sign(grad)
            eps = 1e-4
            with torch.no_grad():
                lp = []
                for sgn in (1.0, -1.0):
                    p = torch.from_numpy(base).to(dev) + sgn * eps * d
                    vv, mm = (p, torch.from_numpy(sc.mu).to(dev)) if name == "v0" else \
                        (torch.from_numpy(sc.v0).to(dev), p)
                    x, _ = rollout(s, H, H.x_rest.clone(), vv, mm, args.adj_steps, checkpoint=0)
                    lp.append(float(H.com_z(x).sum()))
            fd = (lp[0] - lp[1]) / (2 * eps)
            ad = float((grad * d).sum())
            checks[name] = {"direction": "sign(grad)", "eps": eps, "fd": fd, "adjoint": ad,
                            "rel_err": abs(fd - ad) / max(abs(ad), 1e-300)}
        res["fd_check"] = checks
    s.close()
    return {
        "workload": f"{args.adj_scenes} lattices 16x16x8 ({6144 * args.adj_scenes} DOF), "
                    f"{args.adj_steps}-step rollout, checkpoint every 8, d(COM z)/d(v0, mu)",
        "adjoint_solve": {"theta_rel": ADJ_THETA_REL, "l_max": ADJ_L_MAX,
                          "chebyshev_ls_u": list(ADJ_CHEBYSHEV)},
        "launch": {k: tuned[k] for k in ("kernel_variant", "block_threads", "grid")},
        "adjoint_forward_ratio": res["backward_s"] / res["forward_s"],
        **res,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-sweeps", type=int, default=25)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dims", default="128,128,32")
    ap.add_argument("--batch-scenes", type=int, default=4096)
    ap.add_argument("--batch-steps", type=int, default=30)
    ap.add_argument("--per-scene-sample", type=int, default=32)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--adj-scenes", type=int, default=256)
    ap.add_argument("--adj-steps", type=int, default=64)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--sharded-steps", type=int, default=10)
    ap.add_argument("--no-sharded", action="store_true")
    ap.add_argument("--grid-variant", type=int, default=None,
                    help="fix the single scene's launch shape instead of tuning it")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    dims = tuple(int(x) for x in args.dims.split(","))

    from paper_2201_09212_gb300 import scenes
    sc = scenes.terrain_lattice(dims=dims)
    if args.impl == "reference":
        run_reference(args, sc)
        return

    import torch
    ws, rank, local = dist_setup()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the solver has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2201_09212_gb300 import tune, vfpi
    stream = torch.cuda.Stream()
    s = vfpi.Solver.from_scene(sc, theta_th=THETA_TH, l_max=L_MAX, norm="rms", stream=stream)
    s.set_velocity(torch.from_numpy(sc.v0).to(torch.device("cuda", local)))
    if args.grid_variant is not None:            # a fixed launch shape (reproducible captures)
        s.configure_launch(args.grid_variant, 0, 0)
        tuned = {"kernel_variant": args.grid_variant, "block_threads": 0, "grid_ctas": 0,
                 "ms_per_sweep": None, "cached": False}
    else:
        tuned = tune.tune(s, sweeps=30, reps=3)  # launch shape (cached per layout and GPU)
    lay = s.layout()
    stor = s.storage()["storage"]
    dev = torch.device("cuda", local)
    v0 = torch.from_numpy(sc.v0).to(dev)
    x = torch.from_numpy(sc.x0).to(dev)
    torch.cuda.synchronize()

    def step():
        s.set_velocity(v0)
        s.solve_async()
        s.integrate(x)

    for _ in range(args.warmup):
        step()
        s.status()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters, kms = [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
            it, th, _ = s.status()
            iters.append(int(it[0]))
            kms.append(s.last_kernel_ms())
        ev1.record(stream)
        torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    if dist:
        dist.barrier()
    value, elapsed, _ = aggregate(dist, dev, elapsed, sc.n * sum(iters))
    launches_per_step = 3  # warm-start conversion, solve, integrate

    # time to solution of the same step with Chebyshev acceleration (Alg. 3):
    # the sweep is the same kernel, the stop test is reached in fewer sweeps
    s.set_chebyshev(*BATCH_CHEBYSHEV)
    for _ in range(3):
        step()
        s.status()
    cheb_iters = []
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(min(args.steps, 50)):
        step()
        cheb_iters.append(int(s.status()[0][0]))
    ev1.record(stream)
    torch.cuda.synchronize()
    cheb_ms = ev0.elapsed_time(ev1) / len(cheb_iters)
    s.set_chebyshev(0)
    time_to_solution = {"alg1_ms_per_step": 1e3 * elapsed / args.steps,
                        "alg1_iters_per_step": float(np.mean(iters)),
                        "alg3_l_s_u": list(BATCH_CHEBYSHEV), "alg3_ms_per_step": cheb_ms,
                        "alg3_iters_per_step": float(np.mean(cheb_iters))}

    # end to end through the public API with pinned host buffers
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    b_h, phi_h, v_h, x_h = pin(sc.b), pin(sc.phi), pin(sc.v0), pin(sc.x0)
    lam_h = torch.empty(3 * sc.n_c, dtype=torch.float32).pin_memory()
    v_out = torch.empty_like(v_h).pin_memory()
    e2e_iters = []

    def e2e_step():   # one call per time step: inputs up, solve, outputs down, x integrated
        return s.advance(b_h, phi_h, v_h, out_v=v_out, out_lam=lam_h, x=x_h)

    for _ in range(args.warmup):
        e2e_step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_iters.append(e2e_step().iters)
    torch.cuda.synchronize()
    e2e_t = time.perf_counter() - t0
    e2e_value, e2e_t, _ = aggregate(dist, dev, e2e_t, sc.n * sum(e2e_iters))
    h2d = 4 * (sc.n + sc.n_c + sc.n) + 8 * sc.n
    d2h = 4 * (sc.n + 3 * sc.n_c) + 8 * sc.n

    sharded = sharded_one = None
    if ws > 1 and not args.no_sharded:
        sharded = sharded_bench(args, torch, dist, dev, sc, dims, rank, ws)
    elif not args.no_sharded:
        sharded_one = sharded_one_gpu_bench(args, torch, dev, sc, dims,
                                            float(np.mean(kms)) / float(np.mean(iters)))

    batched = None
    if not args.no_batched:
        batched = batched_bench(args, torch, dev, stream, rank)
        batched["env_steps_per_s"], _, _ = aggregate(
            dist, dev, batched["ms_per_env_step"] * batched["steps"] / 1e3,
            args.batch_scenes * batched["steps"])

    adjoint = None
    if not args.no_adjoint and rank == 0:
        adjoint = adjoint_bench(args, torch, dev, stream)

    configs = None
    if not args.no_configs and rank == 0:
        configs = configs_bench(args, torch, dev, stream)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # always the full-BSR count: a compressed storage is reported as an
    # effective fraction next to the measured DRAM bytes, not by a new count
    bps = algorithmic_bytes_per_sweep(sc)
    k_avg = float(np.mean(kms)) / 1e3
    it_avg = float(np.mean(iters))
    achieved = bps * it_avg / k_avg / 1e9
    peak, peak_kind = peaks()
    tr = NCU_TRAFFIC.get((source_hash(), int(tuned["kernel_variant"])))   # only for the captured kernel
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": (tr * it_avg if tr else None),
                # the DRAM bytes the kernel moves (ncu, per launch) over its live time:
                # below frac where v, b, W hit L2, far below it on the 6-value blocks
                "dram_frac": (tr * it_avg / k_avg / 1e9 / peak if tr else None),
                "algorithmic_bytes_per_sweep": bps,
                "kernel": f"k_solve_grid<float,{lay['threads']}> variant {tuned['kernel_variant']}"
                          + STORAGE_NOTE.get(stor, ""),
                "kernel_ms_avg": 1e3 * k_avg}
    cpu = cpu_all = None
    if ws == 1 and not args.no_cpu_baseline:
        rate, cores, dt = cpu_oracle_rate(sc, args.cpu_sweeps)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_sweeps} FP64 oracle V-FPI sweeps of the full workload ({dt:.1f} s)",
               "cpu_model": cpu_model()}
        rate, cores, dt = cpu_oracle_rate_all_cores(sc, dims, 4 * args.cpu_sweeps)
        cpu_all = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": (f"{4 * args.cpu_sweeps} FP64 oracle V-FPI sweeps of each of {cores} "
                              f"z-slabs of the full workload, one process per core, all at once "
                              f"(slowest slab {dt:.1f} s; halo exchange not timed)"),
                   "nproc": os.cpu_count(), "cpu_model": cpu_model()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "dof": sc.n, "blocks": sc.nnzb, "contacts": sc.n_c,
                   "theta_th": THETA_TH, "residual_norm": "rms", "l_max": L_MAX,
                   "iters_per_step": it_avg, "parallelism": "replicas" if ws > 1 else "single",
                   "launch": {"kernel_variant": tuned["kernel_variant"], "ctas": lay["grid"],
                              "threads": lay["threads"], "tuned_ms_per_sweep": tuned["ms_per_sweep"],
                              "from_cache": tuned["cached"]},
                   "l2": ("inputs larger than L2 (" + (
                       f"{((sc.nnzb + sc.n_nodes) // 2) * 40 / 1e6:.0f} MB of upper blocks"
                       if stor == "symmetric"
                       else f"{sc.nnzb * 28 / 1e6:.0f} MB of 6-value blocks" if stor == "blocks6"
                       else f"{sc.nnzb * 40 / 1e6:.0f} MB of blocks") + " streamed per sweep)")},
        "roofline": roofline,
        "time_to_solution": time_to_solution,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "sharded": sharded,
        "sharded_one_gpu": sharded_one,
        "batched": batched,
        "adjoint": adjoint,
        "configs": configs,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    s.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

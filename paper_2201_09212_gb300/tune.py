"""Launch-shape autotuner for the V-FPI solve kernels.

For a solver already built on its problem, ``tune`` times candidate launch
shapes -- for the grid-wide kernel: the kernel variant (threads per CTA, the
CTAs-per-SM register budget, next-chunk prefetch, shared-memory staging of
the chunks by bulk copies with its ring depth, or the symmetric storage of A)
and the number of persistent
CTAs (all that fit, the fewest that keep the same slices per warp, whole
multiples of the SM count); for batched scenes: the threads per CTA of the
CTA-per-scene kernel (warps working on one scene) and the shapes of the
shared-memory-resident cluster kernel (threads per CTA, CTAs per cluster, CTAs
per SM) -- the grid kernel over a fixed number of sweeps, batched scenes over
whole solves at the solver's tolerance (their uneven iteration counts decide
the load balance), on the solver's own problem, timed with CUDA events, and
keeps the fastest (a TMA-ring, symmetric-storage or cluster shape only when it
beats the best plain shape by 2 %, so that timing noise does not switch
kernels from one GPU to the next).  Results
are cached in a JSON file keyed by the layout signature and the GPU name, so a
later solver of the same shape reuses them without timing.
"""
from __future__ import annotations

import json
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "_lib", "tune_cache.json")
# 12..15 need an exactly symmetric A, 28 and 29 (and the scene path's 30) symmetric blocks
GRID_VARIANTS = tuple(range(16)) + (26, 27, 28, 29)
WARPS = {0: 8, 1: 8, 2: 16, 3: 4, 4: 8, 5: 4, 6: 16, 7: 8, 8: 8, 9: 4, 10: 4, 11: 2,
         12: 8, 13: 8, 14: 8, 15: 16, 26: 8, 27: 4, 28: 8, 29: 8}
SCENE_B6 = 30
CLUSTER_VARIANTS = tuple(range(16, 26))
SPECIAL_MARGIN = 0.02


def _signature(solver, gpu: str) -> str:
    lay = solver.layout()
    return f"{gpu}|path{lay['path']}|slices{lay['n_slices']}|slots{lay['slots']}|" \
           f"scenes{solver.n_scenes}|{solver.np_dtype.__name__}"


def _grid_candidates(n_slices, warps, max_grid, sms):
    need = math.ceil(n_slices / warps)
    out = {0}
    k = math.ceil(n_slices / (max_grid * warps))
    out.add(min(max_grid, math.ceil(n_slices / (warps * k))))
    for r in range(1, max_grid // sms + 1):
        out.add(min(need, r * sms))
    return sorted(g for g in out if g == 0 or g <= max_grid)


def _time(solver, sweeps, reps, v_start=None, before_rep=None):
    best = float("inf")
    for _ in range(reps):
        if v_start is not None:
            solver.set_velocity(v_start)
        if before_rep is not None:
            before_rep()
        solver.solve_async()
        solver.status()
        best = min(best, solver.last_kernel_ms())
    return best


def tune(solver, sweeps: int = 20, reps: int = 3, cache: str | None = DEFAULT_CACHE,
         force: bool = False, before_rep=None, condition: str = "") -> dict:
    """Pick and apply the fastest launch shape; returns it with its timings.

    ``before_rep`` (optional) runs before every timed launch -- e.g. a write
    that evicts L2, when the solves it tunes for follow other work; the ranking
    of shapes depends on it (a mid-size scene whose matrix stays in L2 between
    solves prefers other shapes than one that starts each solve from HBM).
    ``condition`` names that setting in the cache key."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = _signature(solver, gpu) + (f"|{condition}" if condition else "")
    table = {}
    if cache and os.path.exists(cache):
        try:
            with open(cache) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
    if key in table and not force:
        best = table[key]
        solver.configure_launch(best["kernel_variant"], best["block_threads"], best["grid_ctas"])
        return dict(best, cached=True)
    lay = solver.layout()
    theta0, lmax0 = solver._theta_th, solver._l_max
    solver.set_tolerance(-1.0, sweeps)
    trials = []
    if lay["path"] == 1:
        for var in GRID_VARIANTS:
            try:
                solver.configure_launch(var, 0, 0)
            except RuntimeError:    # symmetric storage / blocks need A = A^T / symmetric blocks
                continue
            l2 = solver.layout()
            for g in _grid_candidates(l2["n_slices"], WARPS[var], l2["max_grid"], l2["sms"]):
                solver.configure_launch(var, 0, g)
                ms = _time(solver, sweeps, reps, before_rep=before_rep)
                trials.append(dict(kernel_variant=var, block_threads=0, grid_ctas=g,
                                   ms_per_sweep=ms / sweeps, grid=solver.layout()["grid"]))
    else:
        # batched scenes converge after different numbers of sweeps, which
        # decides the load balance: time whole solves at the solver's own
        # tolerance from the same warm start
        solver.set_tolerance(theta0, lmax0)
        v_start = solver.get_velocity()
        shapes = [(v, bt) for v in (0, SCENE_B6) for bt in (64, 128, 256, 512)] + \
            [(v, 0) for v in CLUSTER_VARIANTS]
        for var, bt in shapes:
            try:
                solver.configure_launch(var, bt, 0)
            except RuntimeError:    # shape not available (GPU, asymmetric blocks)
                continue
            ms = _time(solver, sweeps, reps, v_start, before_rep)
            iters, _, _ = solver.status()
            trials.append(dict(kernel_variant=var, block_threads=bt, grid_ctas=0,
                               ms_per_sweep=ms / max(1.0, float(iters.max())), ms_per_solve=ms,
                               grid=solver.layout()["grid"]))
        solver.set_velocity(v_start)
    solver.set_tolerance(theta0, lmax0)
    # the special kernels (TMA ring 8-11 and 26-27, symmetric storage 12-15,
    # cluster 16-25, symmetric blocks 28-30) must beat the best plain shape by
    # SPECIAL_MARGIN: a win inside
    # the timing noise should not switch kernels from one GPU to the next
    cost = lambda t: t.get("ms_per_solve", t["ms_per_sweep"])   # noqa: E731
    plain = [t for t in trials if t["kernel_variant"] < 8]
    best = min(trials, key=cost)
    if plain and best["kernel_variant"] >= 8:
        bp = min(plain, key=cost)
        if cost(best) > (1.0 - SPECIAL_MARGIN) * cost(bp):
            best = bp
    solver.configure_launch(best["kernel_variant"], best["block_threads"], best["grid_ctas"])
    result = dict(best, trials=trials)
    if cache:
        table[key] = {k: best[k] for k in ("kernel_variant", "block_threads", "grid_ctas",
                                           "ms_per_sweep", "grid") if k in best}
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = f"{cache}.{os.getpid()}.tmp"       # several ranks may tune at once
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1)
        os.replace(tmp, cache)
    return dict(result, cached=False)

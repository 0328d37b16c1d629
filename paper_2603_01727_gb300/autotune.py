"""Autotuner of the per-grid launch configuration of a batch of flames.

Two stages, each timed on a small batch of copies of one flame (`copies`
independent simulations under one batch graph), so that the choice reflects
throughput under concurrency, as in a large batch, rather than the latency of
a lone flame:

1. the multigrid fields of sim_params_t: red-black sweeps per smoothing of the
   fused 2D kernels (mg_sweeps, 1 or 2) and the largest level handled by the
   one-block coarse solve (mg_tail_cells), which moves work between the
   one-block coarse kernel and the many-block level kernels.  They change the
   iteration count and the kernel mix, never the stopping test, so every
   candidate converges to the same tolerance;
2. with the best multigrid choice, the cell tile of the projection kernel
   (stage_tile_x: 256 consecutive cells, or a TX x 256/TX tile of cells),
   which sets the blocks' reuse of the pressure's neighbours.  Results do
   not depend on it.

Results are cached per (dim, grid, precision) for the process.
"""

CANDIDATES = ((2, 0), (1, 0), (2, 512), (2, 1024), (2, 16384))
TILE_CANDIDATES = (0, 16, 32, 64)
_cache = {}


def _key(prm):
    dim = int(prm["dim"])
    return dim, tuple(int(v) for v in prm["n"][:dim]), int(prm["precision"])


def time_candidate(prm, geo, fields, sweeps, tail_cells, tile_x=0, copies=8, warmup=8, steps=10, device=None):
    """Milliseconds per batch step of `copies` copies of the flame."""
    import torch
    from .lowmach import Simulation, Batch
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(dev)
    p = dict(prm, mg_sweeps=int(sweeps), mg_tail_cells=int(tail_cells), stage_tile_x=int(tile_x))
    sims = []
    for _ in range(copies):
        s = Simulation(p, geo, device=dev, stream=stream)
        s.set_fields(fields)
        sims.append(s)
    batch = Batch(sims, stream=stream)
    batch.step(warmup)
    batch.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.step(steps)
    e1.record(stream)
    batch.sync()
    ms = e0.elapsed_time(e1) / steps
    batch.close()
    for s in sims:
        s.close()
    return ms


def tune(prm, geo, fields, candidates=CANDIDATES, tiles=TILE_CANDIDATES, copies=8, device=None):
    """(mg_sweeps, mg_tail_cells, stage_tile_x) with the least batch-step time,
    and the table of measured times (ms per step of `copies` flames), keyed by
    the candidate tuple."""
    key = _key(prm)
    if key in _cache:
        return _cache[key]
    table = {}
    for sw, tc in candidates:
        table[(sw, tc, 0)] = time_candidate(prm, geo, fields, sw, tc, 0, copies=copies, device=device)
    best_mg = min(table, key=table.get)
    for tx in tiles:
        cand = (best_mg[0], best_mg[1], tx)
        if cand not in table:
            table[cand] = time_candidate(prm, geo, fields, best_mg[0], best_mg[1], tx, copies=copies,
                                         device=device)
    best = min(table, key=table.get)
    _cache[key] = (best, table)
    return best, table


def apply(prm, choice):
    """Parameters with a tuned (mg_sweeps, mg_tail_cells[, stage_tile_x])."""
    out = dict(prm, mg_sweeps=int(choice[0]), mg_tail_cells=int(choice[1]))
    if len(choice) > 2:
        out["stage_tile_x"] = int(choice[2])
    return out

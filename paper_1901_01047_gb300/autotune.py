"""Autotuner of the submatrix size k_s, the N-update kernel and its tile.

The submatrix method reaches exactly the Markov chain of single-spin updates
for every k_s (DCA++ paper, Sec. 2.3, "Submatrix updates"), and the two
mixed-precision update kernels differ only by rounding, so both are pure
performance parameters.  The tuner times every candidate on the caller's own
walkers, after their warm-up (the orders then have their working size),
with CUDA events on the walker's stream around whole sweeps, and leaves the
walkers on the fastest candidate.  The chains simply continue: each trial
sweep is an ordinary sweep of the run.  After k_s and the kernel, the column
tile of the tensor-core N update (32 or 64 columns of N per tile, for k_s <=
64) is chosen by the device time of the N-update kernel group alone.
"""
import itertools

KS_CANDIDATES = (16, 32, 48, 64, 96, 128)
KERNEL_CANDIDATES = ("tcgen05", "cuda_core")
TILE_CANDIDATES = (64, 32)


def _time_sweeps(gw, sweeps, stream, tries=3):
    """Updates/s over `sweeps` sweeps.  The periodic recompute is the same for
    every candidate, so a trial it falls into is repeated (up to `tries`)."""
    import torch
    for _ in range(tries):
        s = gw.stats()
        p0 = sum(x["proposals"] for x in s)
        r0 = sum(x["recomputes"] for x in s)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gw.sweep(sweeps)
        e1.record(stream)
        e1.synchronize()
        s = gw.stats()
        ms = e0.elapsed_time(e1)
        if sum(x["recomputes"] for x in s) == r0:
            break
    return (sum(x["proposals"] for x in s) - p0) / (ms / 1000.0), ms


def _time_group(gw, group, sweeps):
    """Proposals per second of one kernel group's own device time (CUDA
    events around the group on the walker's stream) over `sweeps` sweeps: the
    column tile changes only the N update, whose share of a whole sweep is
    below the sweep-to-sweep spread of the measurements and recomputes."""
    gw.set_timing([group])
    gw.timing(reset=True)
    p0 = sum(x["proposals"] for x in gw.stats())
    gw.sweep(sweeps)
    t, _ = gw.timing(reset=True)
    props = sum(x["proposals"] for x in gw.stats()) - p0
    gw.set_timing([])
    ms = t[group][0]
    return props / (ms / 1000.0) if ms > 0 else 0.0, ms


def tune(gw, precision, ks_candidates=KS_CANDIDATES, kernels=KERNEL_CANDIDATES, sweeps=2, settle=1):
    """Time each (k_s, kernel) candidate on the walkers `gw` and select the
    fastest.  Returns {"k_sub": .., "update_kernel": .., "table": [...]}.
    `settle` untimed sweeps follow every switch (the first sweep after a
    switch also rebuilds the captured window loop)."""
    import torch
    stream = torch.cuda.current_stream()
    if precision != "mixed":
        kernels = ("cuda_core",)
    table = []
    for ks, kern in itertools.product(ks_candidates, kernels):
        gw.set_tuning(ks, kern)
        if settle:
            gw.sweep(settle)
        rate, ms = _time_sweeps(gw, sweeps, stream)
        table.append({"k_sub": ks, "update_kernel": kern, "updates_per_s": rate, "ms": ms})
    best = max(table, key=lambda r: r["updates_per_s"])
    gw.set_tuning(best["k_sub"], best["update_kernel"])
    tile, tiles = 64, []
    if best["update_kernel"] == "tcgen05" and best["k_sub"] <= 64:
        for bn in TILE_CANDIDATES:
            gw.set_update_tile(bn)
            if settle:
                gw.sweep(settle)
            rate, ms = _time_group(gw, "update", 2 * sweeps)
            tiles.append({"update_tile": bn, "updates_per_s": rate, "ms": ms})
        tile = max(tiles, key=lambda r: r["updates_per_s"])["update_tile"]
        gw.set_update_tile(tile)
    return {"k_sub": best["k_sub"], "update_kernel": best["update_kernel"], "update_tile": tile, "table": table,
            "tiles": tiles}

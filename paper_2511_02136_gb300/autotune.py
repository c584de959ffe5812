"""Launch-shape autotuner for the batched env step (driver over the C ABI).

For a workload it times every candidate launch shape -- warps (envs) per
block; a plain grid, one persistent work-queue launch per capacity class, or
one persistent launch over every class whose warps steal smaller classes'
envs (with the per-class warp split of each block); and env order (as
created, or longest first from a per-env cost estimate) -- with CUDA events
around a caller-supplied run, keeps the fastest, and caches the choice per
workload signature in a JSON file.  The kernels themselves are unchanged: the
shape is set through lob_set_launch / lob_set_multi_split / lob_set_env_costs /
lob_set_threads_per_env / lob_set_tile_records before the timed runs.
Threads per env are 32 (one warp per env) or 64 (one warp per book side, for
the plain step on a plain grid).  The message-tile size (records staged per
copy: 16, 32 or 64) is tuned after the shape: the winning shape is timed
again with each of the other sizes in `tiles`.  The cache records the
threads per env and the tile size with the shape.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, asdict

from . import lob

DEFAULT_CANDIDATES = [(wpb, pers) for pers in (0, 1) for wpb in (1, 2, 4, 8)]
# persistent = 2: one launch over every class (the split derived from the
# classes' env counts for the given warps per block)
MULTI_CANDIDATES = [(wpb, 2) for wpb in (4, 6, 8)]
# two warps per env (one per book side): a plain grid, one env per block
SPLIT_CANDIDATES = [(1, 0, 64)]
# records per staged message tile, timed on the winning shape
TILE_CANDIDATES = (16, 32, 64)


@dataclass
class Choice:
    warps_per_block: int
    persistent: int
    longest_first: bool
    ms: float
    threads_per_env: int = 32
    tile_records: int = 32


def signature(n_envs, caps_hist, mean_msgs, steps, extra=""):
    return f"n{n_envs}|caps{sorted(caps_hist.items())}|m{round(mean_msgs)}|s{steps}|{extra}"


def apply(h, choice: Choice, costs=None):
    lob.lob_set_launch(h, choice.warps_per_block, choice.persistent)
    lob.lob_set_threads_per_env(h, choice.threads_per_env)
    lob.lob_set_tile_records(h, choice.tile_records)
    lob.lob_set_env_costs(h, costs if (choice.longest_first and costs is not None) else None)


def _event_timer(run, repeats):
    """Best of `repeats` CUDA-event timings of run() after one warm-up (ms)."""
    import torch
    run()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune(h, run, costs=None, candidates=DEFAULT_CANDIDATES, repeats=2, cache=None, key=None,
         timer=None, applier=None, timed=None, tiles=(32,)):
    """`run()` performs one timed unit of work on the current stream (it must
    reset/rebind whatever it consumes); returns the fastest Choice.  `timer`
    (run, repeats) -> ms and `applier` (h, choice, costs) default to CUDA
    events and the C ABI; `timed`, a list, receives every candidate timed;
    `tiles` lists the message-tile sizes tried on the winning shape (the
    shapes themselves are timed with 32-record tiles)."""
    timer = timer or _event_timer
    applier = applier or apply
    if cache and key and os.path.exists(cache):
        with open(cache) as f:
            got = json.load(f).get(key)
        if got:
            ch = Choice(**got)
            applier(h, ch, costs)
            return ch
    results = []
    orders = (False, True) if costs is not None else (False,)
    for cand in candidates:
        wpb, pers = cand[0], cand[1]
        tpe = cand[2] if len(cand) > 2 else 32
        for lf in orders:
            if lf and not pers:
                continue          # the order only matters to the work queue
            ch = Choice(wpb, pers, lf, 0.0, threads_per_env=tpe)
            try:
                applier(h, ch, costs)
            except lob.LobError:
                continue          # a shape this handle cannot take (e.g. more classes than warps)
            ch.ms = timer(run, repeats)
            results.append(ch)
    win = min(results, key=lambda c: c.ms)
    for tr in tiles:
        if tr == win.tile_records:
            continue
        ch = Choice(win.warps_per_block, win.persistent, win.longest_first, 0.0,
                    threads_per_env=win.threads_per_env, tile_records=tr)
        try:
            applier(h, ch, costs)
        except lob.LobError:
            continue
        ch.ms = timer(run, repeats)
        results.append(ch)
    if timed is not None:
        timed.extend(results)
    win = min(results, key=lambda c: c.ms)
    applier(h, win, costs)
    if cache and key:
        data = {}
        if os.path.exists(cache):
            with open(cache) as f:
                data = json.load(f)
        data[key] = asdict(win)
        with open(cache, "w") as f:
            json.dump(data, f, indent=1)
    return win

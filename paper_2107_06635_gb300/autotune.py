"""Launch-schedule autotuner of the NTU library.

The library's kernels have schedule choices that change speed but not
results (``ntu_set_tuning``): whether the fused t1 -> t2 kernel pairs its
(k, k') units into one N = 128 product (D = 8), how many ALS CTAs share an SM
(the register budget of the ALS kernel) and on how many CTAs one item's ALS
runs (a thread-block cluster that divides the reduced-metric build).  This
module searches them on the GPU for a given workload by timing the real
batched update with CUDA events (L2 flushed before every timed call), and
keeps the winners in a JSON cache keyed by device name and workload, which
later runs read instead of searching again.

It calls only the library's C ABI (through ``ntu``); nothing here computes
any part of the bond update.
"""
from __future__ import annotations

import itertools
import json
import os
import statistics

from . import ntu

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build",
                             "tuning.json")


AUTOMATIC = {"t12_pair": -1, "als_ctas_per_sm": 0, "als_split": 0, "als_build": 0}


def candidates(D: int, precision: int, split_max: int, builds=(0,)):
    """Every valid tuning of a context: t12 pairing (split-BF16 at D = 8
    only), ALS CTAs per SM, ALS split up to what the context allocated, and
    the ALS reduced-metric builds in `builds` (1 lanes, 2 tensor cores)."""
    pairs = [0, 1] if (D == 8 and precision == ntu.NTU_MIXED_BF16X3) else [-1]
    ctas = [2, 3]
    splits = [s for s in (1, 2, 4) if s <= split_max] if precision != ntu.NTU_FP64 else [1]
    return [{"t12_pair": p, "als_ctas_per_sm": c, "als_split": s, "als_build": b}
            for p, c, s, b in itertools.product(pairs, ctas, splits, builds)]


def builds_of(setter) -> tuple:
    """The reduced-metric builds a context accepts: (1, 2) where the
    tensor-core build is available, else (1,); `setter(**tuning)` applies a
    tuning and raises NTUError when it is refused."""
    try:
        setter(als_build=2)
        return (1, 2)
    except ntu.NTUError:
        return (1,)
    finally:
        setter()


def _timer(torch, stream, flush):
    def timed(fn, reps, warmup=1):
        ts = []
        for i in range(warmup + reps):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if i >= warmup:
                ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)
    return timed


def tune_batch(ctx, n, Ta, Tb, G, Ta_out, Tb_out, info, stream, reps: int = 3):
    """Search the tunings of context `ctx` on its batched update of the n
    device-resident items (torch tensors, `stream` the context's
    torch.cuda.Stream).  Applies the fastest and returns
    {"chosen", "chosen_ms", "automatic_ms", "table": [(tuning, ms), ...]}."""
    import torch
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    timed = _timer(torch, stream, flush)
    run = lambda: ctx.batch_update_dev(n, Ta, Tb, G, Ta_out, Tb_out, info)
    ctx.set_tuning()                                   # automatic choices
    auto_ms = timed(run, reps)
    _, smax = ctx.get_tuning()
    table = []
    builds = builds_of(ctx.set_tuning) if ctx.cfg.precision != ntu.NTU_FP64 else (0,)
    for t in candidates(ctx.D, ctx.cfg.precision, smax, builds):
        ctx.set_tuning(**t)
        table.append((t, timed(run, reps)))
    best, best_ms = min(table, key=lambda x: x[1])
    if best_ms < auto_ms:
        ctx.set_tuning(**best)
        chosen, chosen_ms = best, best_ms
    else:
        ctx.set_tuning()
        chosen, chosen_ms = dict(AUTOMATIC), auto_ms
    ctx.sync()
    return {"chosen": chosen, "chosen_ms": chosen_ms, "automatic_ms": auto_ms,
            "table": [(t, round(ms, 4)) for t, ms in table]}


def tune_uneven(ub, kinds, heaviest: int, stream, reps: int = 3, mode=None):
    """Search the schedule of the uneven batch's critical path: the tuning of
    its heaviest kind (index `heaviest` into `kinds`), with the staged items
    run in `mode` (default: graph replay).  The lighter kinds keep their
    automatic choices.  Applies the fastest; returns the same record as
    tune_batch."""
    import torch
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    timed = _timer(torch, stream, flush)
    mode = ub.GRAPH if mode is None else mode
    run = lambda: ub.run(mode)
    ub.set_tuning(heaviest)
    auto_ms = timed(run, reps)
    D = kinds[heaviest][0]
    table = []
    builds = (builds_of(lambda **t: ub.set_tuning(heaviest, **t))
              if ub.precision != ntu.NTU_FP64 else (0,))
    for t in candidates(D, ub.precision, ub.split_max(heaviest), builds):
        ub.set_tuning(heaviest, **t)
        table.append((t, timed(run, reps)))
    best, best_ms = min(table, key=lambda x: x[1])
    if best_ms < auto_ms:
        ub.set_tuning(heaviest, **best)
        chosen, chosen_ms = best, best_ms
    else:
        ub.set_tuning(heaviest)
        chosen, chosen_ms = dict(AUTOMATIC), auto_ms
    ub.sync()
    return {"kind": list(kinds[heaviest]), "chosen": chosen, "chosen_ms": chosen_ms,
            "automatic_ms": auto_ms, "table": [(t, round(ms, 4)) for t, ms in table]}


def cache_key(device_name: str, workload: dict) -> str:
    return device_name + "|" + json.dumps(workload, sort_keys=True)


def load(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(entries: dict, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(entries, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(device_name: str, workload: dict, path: str = DEFAULT_CACHE):
    """The cached tuning of a workload on this device, or None."""
    return load(path).get(cache_key(device_name, workload))


def remember(device_name: str, workload: dict, tuning: dict, path: str = DEFAULT_CACHE):
    entries = load(path)
    entries[cache_key(device_name, workload)] = tuning
    save(entries, path)

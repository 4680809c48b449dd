"""Autotuner of libws's runtime parameters for one workload.

The paper fixes its launch parameters by a study on its own GPUs (Sec. 5:
thread blocks of 16x16 / 8x8x8, RR = 6 jumps per round).  Here they are picked
per workload by measurement; none of them changes a result, only the time:

  tile_shape           tile shape and threads per tile of the tiled kernels
                       for 2D uint8 images (the library compiles four:
                       SHAPES below; other images have one fixed shape)
  jumps_per_round      pointer hops per pixel per round of step III (RR)
  levels_ctas_per_sm   CTAs per SM of the cooperative waterfall-level kernel

Coordinate descent: each parameter in turn is timed over its candidates with
the others at their best so far (CUDA events on the caller's stream, median of
`reps` runs after one warm-up run).  The chosen values are set on the context
and, with a cache path, stored as JSON keyed by the GPU's name and the caller's
workload key (for instance ndim, dtype, a size bucket and the connectivity), so
a later process applies them without timing.
"""
from __future__ import annotations

import json
import os

SHAPES = {0: "64x32 px / 256 threads", 1: "32x32 px / 256 threads", 2: "128x16 px / 256 threads",
          3: "64x32 px / 512 threads"}
SPACE = {"tile_shape": [0, 1, 2, 3], "jumps_per_round": [2, 4, 6, 8, 12, 16], "levels_ctas_per_sm": [2, 4, 8]}
DEFAULTS = {"tile_shape": 0, "jumps_per_round": 6, "levels_ctas_per_sm": 4}
# the space for workloads without a choice of tile shape (3D, uint16)
SPACE_FIXED_SHAPE = {k: v for k, v in SPACE.items() if k != "tile_shape"}


def size_bucket(n_pixels: int) -> str:
    """Power-of-four bucket of a pixel count (workloads within 4x share settings)."""
    b = 0
    while (1 << (2 * (b + 1))) <= max(int(n_pixels), 1):
        b += 1
    return f"4^{b}"


def _median(xs):
    s = sorted(xs)
    return s[len(s) // 2]


def descend(time_fn, space=None, start=None):
    """Coordinate descent over `space` ({name: [candidates]}) with a timing
    function time_fn(params) -> ms.  Returns (best params, best ms, table of
    (params, ms) in the order measured).  Pure host logic."""
    space = SPACE if space is None else space
    best = dict(DEFAULTS if start is None else start)
    for k in space:
        best.setdefault(k, space[k][0])
    table = []
    best_ms = None
    for name, cands in space.items():
        scores = {}
        for v in cands:
            p = dict(best, **{name: v})
            ms = time_fn(p)
            table.append((p, ms))
            scores[v] = ms
        v_best = min(cands, key=lambda v: (scores[v], cands.index(v)))
        best[name] = v_best
        best_ms = scores[v_best]
    return best, best_ms, table


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def autotune(ctx, run, key: str, reps: int = 5, space=None, cache_path: str | None = None, stream=None):
    """Tunes `ctx` for the work `run()` enqueues (any libws call sequence on the
    current stream).  Returns {"params", "ms", "table", "cached"}; the chosen
    params stay set on the context (its other tuning fields back at their
    defaults).  A CUDA graph captures the parameters in force when it is
    created, so tune before capturing."""
    import torch
    dev = torch.cuda.get_device_name(torch.cuda.current_device())
    ckey = f"{dev}|{key}"
    if cache_path:
        cache = _load_cache(cache_path)
        if ckey in cache:
            params = cache[ckey]["params"]
            ctx.set_tuning(**params)
            return {"params": params, "ms": cache[ckey]["ms"], "table": [], "cached": True}
    stream = torch.cuda.current_stream() if stream is None else stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def time_fn(params):
        ctx.set_tuning(**params)
        run()
        ctx.check()
        ts = []
        for _ in range(reps):
            e0.record(stream)
            run()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ctx.check()
        return _median(ts)

    best, best_ms, table = descend(time_fn, space)
    ctx.set_tuning(**best)
    if cache_path:
        cache = _load_cache(cache_path)
        cache[ckey] = {"params": best, "ms": best_ms}
        tmp = f"{cache_path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return {"params": best, "ms": best_ms, "table": [(p, round(ms, 4)) for p, ms in table], "cached": False}

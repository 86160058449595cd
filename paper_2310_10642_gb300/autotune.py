"""Picks the tile sizes, the per-tile batch depth and the number of view
groups of a frame by timing.

Three launch-shape knobs change speed but not results: ``tile_size`` (16 or
32, the side of the square compositing tiles, one thread block each),
``bin_size`` (16, 32 or 64, a multiple of ``tile_size``: the side of the
binning tiles whose depth-ordered lists the sort builds) and ``batch_depth``
(how many splat records a block stages in shared memory per batch).  Which
combination is fastest depends on the splat-size distribution and the image
sizes, so ``tune`` renders the caller's own frame (forward + backward) with
every candidate, times it with CUDA events, and returns the fastest.  Results are cached in a JSON file keyed
by the device and the shape of the workload, so a training loop tunes once.

``tune_groups`` then times the whole step as one batch against the views as
two (or more) groups on their own streams (``render.SplitFrame``): that
overlap pays when every group still has enough views to keep the GPU busy.

Cache file: ``$FGS4D_AUTOTUNE_CACHE`` if set, else
``~/.cache/fgs4d/autotune.json``; ``cache=None`` disables it.
"""
from __future__ import annotations

import json
import os
import statistics
from typing import Callable

TILE_SIZES = (16, 32)
BIN_FACTORS = (1, 2, 4)  # binning tile side / compositing tile side
MAX_BIN = 64
BATCH_DEPTHS = (64, 128, 256)
KNOBS = ("tile_size", "bin_size", "batch_depth")


def default_cache_path() -> str:
    return os.environ.get("FGS4D_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "fgs4d", "autotune.json"))


def candidates(tiles=TILE_SIZES, depths=BATCH_DEPTHS, factors=BIN_FACTORS) -> list:
    return [dict(tile_size=t, bin_size=t * f, batch_depth=b) for t in tiles for f in factors if t * f <= MAX_BIN
            for b in depths]


def workload_key(device_name: str, n: int, views: list, sh_degree: int, n_freq: int, record_fp16: int,
                 shs_bf16: bool) -> str:
    """Signature of what the timing depends on: the device, the number of
    Gaussians (to two significant digits), the multiset of image sizes, the
    4DSH size and the storage precision."""
    n2 = int(float(f"{max(int(n), 1):.2g}"))
    sizes = {}
    for v in views:
        wh = f"{int(v['width'])}x{int(v['height'])}"
        sizes[wh] = sizes.get(wh, 0) + 1
    vs = ",".join(f"{k}*{sizes[k]}" for k in sorted(sizes))
    return (f"{device_name}|n~{n2}|views={vs}|L={int(sh_degree)}|K={int(n_freq)}|"
            f"rec16={int(record_fp16)}|shs16={int(bool(shs_bf16))}")


def load_cache(path: str | None) -> dict:
    if not path or not os.path.exists(path):
        return {}
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(path: str | None, key: str, entry: dict) -> None:
    if not path:
        return
    d = load_cache(path)
    d[key] = entry
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def select(timings: list) -> dict:
    """The fastest candidate of [(candidate, ms), ...]; ties go to the earlier one."""
    if not timings:
        raise ValueError("no candidate was timed")
    best = min(range(len(timings)), key=lambda i: (timings[i][1], i))
    return dict(timings[best][0])


def tune_with(timer: Callable[[dict], float], cands: list, key: str, cache: str | None) -> tuple:
    """Host logic of ``tune``: cached choice if present, else time every
    candidate with ``timer(candidate) -> ms``.  Returns (choice, table)."""
    hit = load_cache(cache).get(key)
    if hit and all(k in hit.get("choice", {}) for k in KNOBS):
        return dict(hit["choice"]), hit.get("table", [])
    table = [(dict(c), float(timer(c))) for c in cands]
    choice = select(table)
    store_cache(cache, key, dict(choice=choice, table=[dict(c, ms=round(ms, 4)) for c, ms in table]))
    return choice, [dict(c, ms=round(ms, 4)) for c, ms in table]


def tune(params: dict, views: list, options: dict | None = None, cands: list | None = None, reps: int = 3,
         warmup: int = 2, cache: str | None = "default") -> tuple:
    """Fastest (tile_size, bin_size, batch_depth) for rendering ``params`` into ``views``
    forward and backward.  Returns (options with the choice filled in, table
    of candidate timings in ms per forward+backward).  Runs the frame
    ``(warmup + reps) x len(cands)`` times."""
    import torch

    from . import render as R

    opts = dict(options or {})
    cands = cands or candidates()
    cache = default_cache_path() if cache == "default" else cache
    n = int(params["logit"].shape[0])
    key = workload_key(torch.cuda.get_device_name(), n, views, params["sh_degree"], params["n_freq"],
                       opts.get("record_fp16", 0), params["shs"].dtype == torch.bfloat16)
    stream = torch.cuda.current_stream()

    def timer(c: dict) -> float:
        fr = R.Frame(n, views, dict(opts, **c))
        fr.forward(params, check=True)
        gen = torch.Generator(device=fr.device).manual_seed(0)
        dL = torch.randn(3 * fr.total_pixels, device=fr.device, generator=gen)
        grads = {k: torch.empty(params[k].shape, device=fr.device, dtype=torch.float32) for k in R.PARAM_KEYS}

        def step():
            fr.forward(params, check=False)
            fr.backward(params, dL, grads)

        for _ in range(warmup):
            step()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        del fr, dL, grads
        torch.cuda.empty_cache()
        return statistics.median(times)

    choice, table = tune_with(timer, cands, key, cache)
    return dict(opts, **choice), table


def tune_groups(params: dict, views: list, options: dict, groups=(1, 2), reps: int = 3, warmup: int = 2) -> tuple:
    """Fastest number of view groups for the forward + backward step of
    ``params`` into ``views`` with ``options`` (a launch shape from ``tune``):
    1 is one Frame on one stream, g > 1 a SplitFrame of g groups.  Returns
    (groups, table of [groups, ms])."""
    import torch

    from . import render as R

    n = int(params["logit"].shape[0])
    stream = torch.cuda.current_stream()
    table = []
    for g in groups:
        fr = R.SplitFrame(n, views, options, groups=g) if g > 1 else R.Frame(n, views, options)
        fr.forward(params, check=True)
        gen = torch.Generator(device=fr.device).manual_seed(0)
        dL = torch.randn(3 * fr.total_pixels, device=fr.device, generator=gen)
        grads = {k: torch.empty(params[k].shape, device=fr.device, dtype=torch.float32) for k in R.PARAM_KEYS}
        for _ in range(warmup):
            fr.step(params, dL, grads)
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fr.step(params, dL, grads)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        table.append((dict(groups=int(g)), statistics.median(times)))
        del fr, dL, grads
        torch.cuda.empty_cache()
    best = select(table)
    return best["groups"], [dict(c, ms=round(ms, 4)) for c, ms in table]

"""Tile autotuner for the fused step (single lattice or batch).

Times each candidate thread-block tile for a few steps on the caller's own
state (CUDA events on the current stream), keeps the fastest, and caches the
choice per (GPU, lattice, precision, problem size class) in a JSON file next
to the built library.  Results never depend on the tile, so tuning is safe on
a live state; the steps it takes advance the state.
"""
import json
import os

from . import build as _build

CACHE = os.path.join(_build.BUILD, "tiles.json")

CANDIDATES = {
    # (lattice dimension, the step kernel's largest block): tiles; every
    # lattice and precision has an entry (the float and half kernels are
    # built for 128 threads, the double ones for 256)
    (1, 128): [(128, 1, 1), (64, 1, 1), (96, 1, 1), (32, 1, 1)],
    (1, 256): [(256, 1, 1), (128, 1, 1), (64, 1, 1), (32, 1, 1)],
    (2, 128): [(64, 2, 1), (32, 4, 1), (16, 8, 1), (128, 1, 1), (32, 2, 1), (64, 1, 1)],
    (2, 256): [(64, 4, 1), (32, 8, 1), (128, 2, 1), (64, 2, 1), (32, 4, 1)],
    (3, 256): [(32, 4, 2), (32, 2, 4), (64, 2, 2), (32, 8, 1), (16, 8, 2), (32, 4, 1)],
    (3, 128): [(16, 8, 1), (32, 4, 1), (32, 2, 2), (16, 4, 2), (64, 2, 1)],
}


def _gpu_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _load():
    try:
        return json.load(open(CACHE))
    except (OSError, ValueError):
        return {}


def _save(d):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp%d" % os.getpid()
    json.dump(d, open(tmp, "w"), indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _size_class(nodes):
    return "2^%d" % max(0, int(nodes).bit_length() - 1)


def tune(obj, lattice_d, precision, nodes, kind, steps=40, use_cache=True):
    """Choose a tile for `obj` (a Simulation or a Batch: set_tile, step).
    Returns (tile, {tile: seconds per step})."""
    import torch
    from . import tile_limit
    maxthr = tile_limit(lattice_d, precision)
    key = "|".join([_gpu_name(), "D%d" % lattice_d, precision, kind, _size_class(nodes)])
    cache = _load() if use_cache else {}
    if key in cache:
        tile = tuple(cache[key]["tile"])
        obj.set_tile(*tile)
        return tile, {tuple(int(v) for v in k.split("x")): t for k, t in cache[key]["times"].items()}
    times = {}
    stream = torch.cuda.current_stream()
    for tile in CANDIDATES[(lattice_d, maxthr)]:
        try:
            obj.set_tile(*tile)
        except Exception:
            continue
        obj.step(4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        obj.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        times[tile] = e0.elapsed_time(e1) / 1e3 / steps
    best = min(times, key=times.get)
    obj.set_tile(*best)
    cache = _load()
    cache[key] = {"tile": list(best), "times": {"x".join(map(str, k)): v for k, v in times.items()}}
    _save(cache)
    return best, times

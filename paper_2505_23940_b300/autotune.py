"""Autotuner of the library's launch parameters (fs_set_tuning).

For one grid it times a few steps per candidate value with CUDA events on a
copy of the state, one parameter at a time (coordinate search, the others held
at their best so far), and caches the winner per grid shape and precision in a
JSON file (FS_TUNE_CACHE, default ~/.cache/fsstep_tuning.json).  Results do not
depend on these parameters; only speed does.
"""
import json
import os

import torch

CANDIDATES = {
    "stencil_bx": [32, 64, 128],
    "fft_lines": [4, 8, 16],
    "predictor_cells": [4, 2],
    "predictor_zmarch": [8, 4, 1],
    "ysolve_segments": [4, 8, 16],
}


def cache_path():
    return os.environ.get("FS_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "fsstep_tuning.json"))


def shape_key(grid):
    return "%dd-%dx%dx%d-%s" % (grid.dim, grid.n[0], grid.n[1], grid.n[2],
                                "fp64" if grid.dtype == torch.float64 else "mixed")


def _load():
    try:
        return json.load(open(cache_path()))
    except Exception:
        return {}


def _save(data):
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + ".tmp"
        json.dump(data, open(tmp, "w"), indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass


def apply(grid, params):
    for k, v in params.items():
        grid.set_tuning(k, v)


def _time(grid, u, dt, body, steps):
    uu = [x.clone() for x in u]
    bb = body.clone() if body is not None else None
    grid.step(uu, dt, 1, body=bb)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(grid.stream)
    grid.step(uu, dt, steps, body=bb)
    e1.record(grid.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def tune(grid, u, dt, body=None, steps=3, use_cache=True):
    """Pick the launch parameters of `grid`; returns {key: value} (also applied)."""
    key = shape_key(grid)
    data = _load() if use_cache else {}
    if key in data:
        apply(grid, data[key])
        return data[key]
    best = {k: 0 for k in CANDIDATES}
    apply(grid, best)
    best_t = _time(grid, u, dt, body, steps)
    for k, values in CANDIDATES.items():
        for v in values:
            trial = dict(best, **{k: v})
            apply(grid, trial)
            t = _time(grid, u, dt, body, steps)
            if t < best_t:
                best, best_t = trial, t
        apply(grid, best)
    if use_cache:
        data = _load()
        data[key] = best
        _save(data)
    return best

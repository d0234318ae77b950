"""Autotuner of the blend schedule: tile shape, pixels per thread (forward and
backward), Gaussians staged per batch, the persistent-grid size and whether the
tile lists take the occlusion cut.

None of these choices changes forward results (the per-pixel 3-sigma test is
explicit, so tiles are only a conservative cover, and the occlusion cut drops only
pairs no pixel reaches); they change only the summation order of atomically
accumulated gradients. The tuner times a
forward + backward of the caller's own workload with CUDA events and keeps the
fastest option set, by coordinate descent from the caller's base schedule (the
library defaults unless one is given). Results
are cached in a JSON file keyed by a workload signature.
"""
from __future__ import annotations

import json
import os
import statistics

import torch

from . import binding as B

__all__ = ["SEARCH_SPACE", "signature", "autotune", "options_from_dict", "options_to_dict"]

SEARCH_SPACE = {
    "tile": [(16, 16), (16, 8), (32, 8), (8, 8)],
    "pixels_per_thread": [1, 2, 4],
    "bwd_pixels_per_thread": [1, 2, 4],
    "batch": [64, 128, 256, 512],
    "blocks_per_sm": [0, 2, 4, 8, 12, 16],
    "full_lists": [0, 1],
}
FIELDS = ("tile_w", "tile_h", "pixels_per_thread", "bwd_pixels_per_thread", "batch", "blocks_per_sm", "full_lists")


def options_to_dict(o: B.Options) -> dict:
    return {k: int(getattr(o, k)) for k in FIELDS}


def options_from_dict(d: dict, base: B.Options | None = None) -> B.Options:
    o = B.s3gs_options_default() if base is None else B.Options.from_buffer_copy(base)
    for k in FIELDS:
        if k in d:
            setattr(o, k, int(d[k]))
    return o


def _valid(o: B.Options) -> bool:
    px = o.tile_w * o.tile_h
    for p in (o.pixels_per_thread or 2, o.bwd_pixels_per_thread or 4):
        if (px // p) % 32 != 0 or px % p != 0:
            return False
    return True


def signature(params: dict, cameras, options: B.Options) -> str:
    """Workload key: Gaussian count (to 2 significant digits), SH degree, view sizes
    and the modes that change the kernels (deterministic, recompute)."""
    n = int(params["means"].shape[0])
    n2 = float(f"{n:.2g}")
    sizes = sorted({f'{c["width"]}x{c["height"]}' for c in cameras})
    return (f"n{n2:g}-sh{params['sh_degree']}-v{len(cameras)}-{'+'.join(sizes)}"
            f"-det{options.deterministic}-rec{options.recompute}")


def _time(renderer, params, cameras, opt, grads_in, repeats):
    out = renderer.forward(params, cameras, options=opt)
    g = renderer.backward(params, len(cameras), grads_in)
    torch.cuda.synchronize()
    times = []
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        renderer.forward(params, cameras, options=opt, outputs=out)
        renderer.backward(params, len(cameras), grads_in, into=g)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def autotune(renderer, params: dict, cameras, base: B.Options | None = None, cache_path: str | None = None,
             repeats: int = 3, rounds: int = 2, verbose: bool = False) -> B.Options:
    """Return the fastest option set for this workload (and cache it)."""
    base = B.s3gs_options_default() if base is None else base
    key = signature(params, cameras, base)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        return options_from_dict(cache[key]["options"], base)

    P = sum(int(c["width"]) * int(c["height"]) for c in cameras)
    gen = torch.Generator(device=renderer.device).manual_seed(0)
    grads_in = {k: torch.randn(n, device=renderer.device, generator=gen)
                for k, n in (("rgb", 3 * P), ("depth", P), ("pointmap", 3 * P), ("alpha", P))}
    best = options_from_dict({}, base)
    best.tile_w, best.tile_h = best.tile_w or 16, best.tile_h or 16
    best_t = _time(renderer, params, cameras, best, grads_in, repeats)
    tried = {json.dumps(options_to_dict(best), sort_keys=True): best_t}
    for _ in range(rounds):
        improved = False
        for dim, values in SEARCH_SPACE.items():
            for val in values:
                cand = options_from_dict(options_to_dict(best), base)
                if dim == "tile":
                    cand.tile_w, cand.tile_h = val
                else:
                    setattr(cand, dim, val)
                if not _valid(cand):
                    continue
                sig = json.dumps(options_to_dict(cand), sort_keys=True)
                if sig in tried:
                    continue
                t = _time(renderer, params, cameras, cand, grads_in, repeats)
                tried[sig] = t
                if verbose:
                    print(f"autotune {sig} {t:.3f} ms")
                if t < best_t:
                    best, best_t, improved = cand, t, True
        if not improved:
            break
    if cache_path:
        cache[key] = {"options": options_to_dict(best), "ms_fwd_bwd": best_t, "candidates_timed": len(tried)}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return best

"""Autotuner for the rendering schedule: tile shape (8x8, 16x16, 32x8) and
radix-sort keys per CTA (2048, 4096, 8192).  Neither changes any result; the
tuner times a few graph-captured training steps (forward + loss + backward,
all through librogs) of each candidate on representative frames and keeps
the fastest.  Choices are cached in a JSON file keyed by the set of view
shapes, the number of semantic classes and the map size (power-of-two
bucket)."""
from __future__ import annotations

import json
import math
import os
from typing import Dict, List, Sequence, Tuple

import torch

from . import render as R

TILES = ((16, 16), (32, 8), (8, 8))
SORT_TILES = (2048, 4096, 8192)


def cache_key(cams: Sequence, num_classes: int, n_surfels: int) -> str:
    shapes = sorted({(int(c.kind), int(c.width), int(c.height)) for c in cams})
    bucket = int(math.ceil(math.log2(max(n_surfels, 1))))
    return f"C{num_classes}|N2^{bucket}|V{len(cams)}|" + ",".join(f"{k}:{w}x{h}" for k, w, h in shapes)


def _time_candidate(m: R.SurfelTensors, frames_cams: List[list], exposure, targets, num_classes, tile, sort_tile,
                    record_capacity, pair_capacity, steps) -> float:
    rr = R.Renderer(num_classes, record_capacity=record_capacity, pair_capacity=pair_capacity, tile=tile,
                    sort_tile=sort_tile)
    try:
        frames = [rr.frame(c) for c in frames_cams]
        loss = torch.empty(1, device="cuda")
        grads = R.zero_grads(m, exposure)
        for fr in frames:
            rr.forward(m, fr, exposure)
        torch.cuda.synchronize()
        for fr in frames:
            rr.counts(fr)
        graphs = [rr.train_graph(m, fr, exposure, *tg, loss, grads) for fr, tg in zip(frames, targets)]
        for g in graphs:
            g.launch()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(steps):
            graphs[k % len(graphs)].launch()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        for g in graphs:
            g.close()
        return ms
    finally:
        rr.close()


def tune(m: R.SurfelTensors, frames_cams: List[list], exposure, targets, num_classes: int,
         record_capacity: int, pair_capacity: int, steps: int = 6, cache_path: str = None,
         tiles=TILES, sort_tiles=SORT_TILES) -> Tuple[dict, Dict[str, float]]:
    """Returns ({"tile": (w, h), "sort_tile": s}, {candidate: ms per step}).
    `targets` holds (rgb, label, mask) device tensors per frame.  Must run on
    a non-default stream (graph capture)."""
    key = cache_key(frames_cams[0], num_classes, m.n)
    if cache_path and os.path.exists(cache_path):
        cache = json.load(open(cache_path))
        if key in cache:
            c = cache[key]
            return {"tile": tuple(c["tile"]), "sort_tile": c["sort_tile"]}, c.get("timings", {})
    timings = {}
    for tile in tiles:
        for st in sort_tiles:
            timings[f"{tile[0]}x{tile[1]}/{st}"] = _time_candidate(m, frames_cams, exposure, targets, num_classes,
                                                                    tile, st, record_capacity, pair_capacity, steps)
    best = min(timings, key=timings.get)
    tw, th = best.split("/")[0].split("x")
    choice = {"tile": (int(tw), int(th)), "sort_tile": int(best.split("/")[1])}
    if cache_path:
        cache = json.load(open(cache_path)) if os.path.exists(cache_path) else {}
        cache[key] = {"tile": list(choice["tile"]), "sort_tile": choice["sort_tile"], "timings": timings}
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        json.dump(cache, open(cache_path, "w"), indent=1)
    return choice, timings

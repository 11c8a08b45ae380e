"""Tile-shape autotuner for the migration kernel and the batched launch.

A CTA of the migration kernel owns cx x cy image columns and cz groups of 16 depths
(cx * cy * cz = 256 threads).  The shape trades the aperture cull and time-window length
(compact footprints) against the range of the v(z) delta evaluation (tall or wide tiles need
the 20-term ln(1 + rho) fit or are refused).  The tuner times every candidate on the job's
own geometry with CUDA events on the current stream and caches the fastest in a JSON file
keyed by (trace precision, nt bucket, grid bucket, velocity kind), so that jobs of one bucket
are timed once per machine.
"""
from __future__ import annotations

import json
import math
import os
import tempfile
from typing import Dict, List, Optional, Tuple

import torch

from . import kirchhoff as kh

Tile = Tuple[int, int, int]

CANDIDATES: Dict[int, List[Tile]] = {
    3: [(16, 16, 1), (32, 8, 1), (16, 8, 2), (8, 8, 4), (8, 4, 8), (64, 4, 1)],
    2: [(64, 1, 4), (32, 1, 8), (128, 1, 2), (16, 1, 16), (256, 1, 1)],
}

_PREC = {torch.float32: "f32", torch.float16: "f16", torch.bfloat16: "bf16"}


def default_cache_path() -> str:
    return os.environ.get("KH_TILE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "kirchhoff_gb300", "tiles.json"))


def bucket_key(survey, trace_dtype=torch.float32) -> str:
    """(precision, nt bucket, grid bucket, velocity kind): nt rounded up to a power of two,
    each grid dimension rounded up to 32 samples, the grid spacing to a quarter octave (the
    tile's extent in metres decides its v(z) fit length and cull)."""
    nt_b = 1 << max(0, math.ceil(math.log2(max(int(survey.nt), 1))))
    ny = survey.ny if survey.dim == 3 else 1
    grid = "x".join(str(-(-int(v) // 32) * 32) for v in (survey.nx, ny, survey.nz))
    h_b = 2.0 ** (round(4.0 * math.log2(max(float(survey.dx), 1e-6))) / 4.0)
    vel = survey.vel if (survey.vel != "linear" or survey.k != 0.0) else "const"
    return f"{_PREC[trace_dtype]}|nt{nt_b}|g{grid}|h{h_b:.4g}|{vel}|{survey.weight}|d{survey.dim}"


class TileTuner:
    """Chooses and sets a plan's tile (``Plan.set_tile``), timing candidates on a prefix of
    at most ``sample_traces`` of the job's traces, ``reps`` timed runs after one warm-up."""

    def __init__(self, path: Optional[str] = None, sample_traces: int = 4000, reps: int = 2,
                 candidates: Optional[Dict[int, List[Tile]]] = None):
        self.path = path or default_cache_path()
        self.sample_traces = sample_traces
        self.reps = reps
        self.candidates = candidates or CANDIDATES
        self.cache: Dict[str, Dict] = {}
        self.timed = 0          # candidate timings run by this tuner (cache misses)
        if os.path.exists(self.path):
            with open(self.path) as f:
                self.cache = json.load(f)

    def _save(self):
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d or ".", suffix=".tmp")
        with os.fdopen(fd, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def time_tile(self, plan: "kh.Plan", hdr: "kh.Headers", traces, tile: Tile) -> Optional[float]:
        """Milliseconds per migrate of the sample with ``tile``; None if the plan refuses it."""
        m = min(hdr.ntr, self.sample_traces)
        sub = kh.Headers(hdr.sx[:m], hdr.sy[:m], hdr.rx[:m], hdr.ry[:m], device=traces.device)
        d = traces[:m].contiguous()
        out = torch.empty(plan.image_shape, dtype=torch.float32, device=traces.device)
        plan.set_tile(tile)
        try:
            plan.migrate(sub, d, out)
        except kh.KirchhoffError as e:
            if e.status == kh.KH_ERR_UNSUPPORTED:
                return None
            raise
        st = torch.cuda.current_stream()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(self.reps):
            plan.migrate(sub, d, out)
        b.record(st)
        b.synchronize()
        self.timed += 1
        return a.elapsed_time(b) / self.reps

    def choose(self, plan: "kh.Plan", hdr: "kh.Headers", traces) -> Tile:
        """Sets and returns the cached or fastest tile for the plan's bucket."""
        key = bucket_key(plan.survey, plan.trace_dtype)
        hit = self.cache.get(key)
        if hit is not None:
            tile = tuple(hit["tile"])
            plan.set_tile(tile)
            return tile
        results = {}
        for c in self.candidates[plan.survey.dim]:
            ms = self.time_tile(plan, hdr, traces, c)
            if ms is not None:
                results[c] = ms
        if not results:
            raise kh.KirchhoffError(kh.KH_ERR_UNSUPPORTED, f"no tile candidate runs for {key}")
        best = min(results, key=results.get)
        plan.set_tile(best)
        self.cache[key] = {"tile": list(best), "ms": {f"{c[0]}x{c[1]}x{c[2]}": v for c, v in results.items()}}
        self._save()
        return best

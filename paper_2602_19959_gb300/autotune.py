"""Autotuner for the batched (graph-captured) launch.

A launch's schedule has two kinds of free parameters:
  * the plan: how many events the UNet processes per pass (chunk_events). Small chunks
    keep a pass's activations resident in the 129 MB L2 and shrink the pool; large chunks
    give each layer kernel more tiles per SM and fewer launches;
  * the grids: how many CTAs per SM each persistent kernel family launches (pvf_schedule:
    the front, whose grid sets the events each CTA walks and, in the tensor-core forms,
    the FC tile (passes of 256 tracks at 1-2 CTAs per SM, 128 at 3-4), the six tensor-core conv
    kernels, whose grids set the tiles per CTA, and the peak finder). More resident CTAs
    hide latency; fewer leave each CTA more shared-memory and register headroom and
    shorten the tail of the last wave.
For a workload the tuner captures the whole batch as one CUDA graph per candidate, times
graph launches with CUDA events (L2 flushed between launches), and walks the parameters
one at a time (coordinate descent), keeping each parameter at its fastest value before
moving to the next. The result is a table of the schedule plus every trial, which
PVFinder(schedule=...) and pvf_create read; results never depend on the schedule.
"""

from __future__ import annotations

import json
import os

FAMILIES = ("front", "enc2", "enc3", "enc4_up3", "dec3_up2", "dec2_up1", "dec1_final", "tail")
# CTAs per SM tried for each family (0 = as many as fit; the library clamps larger values)
GRID_CANDIDATES = {"front": (1, 2, 3, 4), "enc2": (2, 3, 4, 6), "enc3": (1, 2, 3, 4), "enc4_up3": (1,),
                   "dec3_up2": (1,), "dec2_up1": (1, 2), "dec1_final": (2, 3, 4, 5),
                   "tail": (1, 2, 4, 8)}
TUNED_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned")


def _time_graph(pv, feats, offs, repeats, warmup, flush):
    import torch
    out = pv.alloc_outputs(int(offs.numel() - 1))
    g = pv.capture_graph(feats, offs, out)
    for _ in range(warmup):
        g.launch()
    times = []
    for _ in range(repeats):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.launch()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    g.close()
    return min(times)


def tune(weights, batch, precision="bf16", chunk_candidates=(0,), repeats=3, warmup=1, max_pv=64,
         fp8_act_scales=None, flush_mb=512, passes=1, log=None):
    """Coordinate descent over chunk_events and the CTAs per SM of each kernel family.
    Returns (best: dict with "chunk_events" and the schedule, trials: list of dicts)."""
    import torch
    from .pvf import PVFinder

    n = batch.n_events
    feats = torch.from_numpy(batch.features).cuda()
    offs = torch.from_numpy(batch.offsets).cuda()
    flush = torch.empty(flush_mb * 1024 * 1024, dtype=torch.uint8, device="cuda")
    trials = []
    cache = {}

    def measure(chunk, sched):
        key = (chunk, tuple(sorted(sched.items())))
        if key in cache:
            return cache[key]
        pv = PVFinder(weights, precision=precision, max_events=n, chunk_events=min(chunk, n) if chunk else 0,
                      max_pv_per_event=max_pv, fp8_act_scales=fp8_act_scales, schedule=sched)
        ms = _time_graph(pv, feats, offs, repeats, warmup, flush)
        pv.close()
        del pv
        torch.cuda.empty_cache()
        trials.append({"chunk_events": chunk, **sched, "ms": ms})
        if log:
            log(f"chunk {chunk or n} {sched}: {ms:.3f} ms")
        cache[key] = ms
        return ms

    chunk, sched = 0, {f: 0 for f in FAMILIES}
    best_ms = measure(chunk, sched)
    for _ in range(passes):
        for c in chunk_candidates:
            ms = measure(c, sched)
            if ms < best_ms:
                best_ms, chunk = ms, c
        for fam in FAMILIES:
            for v in GRID_CANDIDATES[fam]:
                cand = dict(sched, **{fam: v})
                ms = measure(chunk, cand)
                if ms < best_ms:
                    best_ms, sched = ms, cand
    best = {"chunk_events": chunk, **sched, "ms": best_ms}
    return best, trials


def table_path(precision: str, workload: str) -> str:
    return os.path.join(TUNED_DIR, f"{precision}_{workload}.json")


def save_table(path, workload: str, precision: str, best: dict, trials: list, default_ms: float):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as fh:
        json.dump({"workload": workload, "precision": precision, "default_ms": default_ms,
                   "best": best, "trials": trials}, fh, indent=1)


def load_schedule(path):
    """(chunk_events, schedule dict) of a saved table."""
    with open(path) as fh:
        best = json.load(fh)["best"]
    return int(best.get("chunk_events", 0)), {f: int(best.get(f, 0)) for f in FAMILIES}

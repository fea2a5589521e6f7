"""Autotuner for the batched (graph-captured) launch.

The free parameter of a launch is its schedule: how many events the UNet processes per
pass (chunk_events). Small chunks keep a pass's activations resident in the 129 MB L2
and need a smaller pool; large chunks give each layer kernel more tiles per SM and fewer
launches. For a given workload the tuner captures one CUDA graph per candidate chunk
size, times graph launches with CUDA events (L2 flushed between launches) and returns
the fastest, with the whole table.
"""

from __future__ import annotations

import json


def tune_chunk(weights, batch, precision="bf16", candidates=(128, 256, 512, 1024, 2048, 0),
               repeats=5, warmup=2, max_pv=64, fp8_act_scales=None, flush_mb=512, log=None):
    """Returns (best_chunk, {chunk: ms per launch}). chunk 0 = the whole batch at once."""
    import torch
    from .pvf import PVFinder

    n = batch.n_events
    feats = torch.from_numpy(batch.features).cuda()
    offs = torch.from_numpy(batch.offsets).cuda()
    flush = torch.empty(flush_mb * 1024 * 1024, dtype=torch.uint8, device="cuda")
    table = {}
    for c in candidates:
        if c and c >= n and 0 in candidates:
            continue                      # same schedule as the whole batch
        pv = PVFinder(weights, precision=precision, max_events=n, chunk_events=min(c, n) if c else 0,
                      max_pv_per_event=max_pv, fp8_act_scales=fp8_act_scales)
        out = pv.alloc_outputs(n)
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
        table[c] = min(times)
        if log:
            log(f"chunk {c or n}: {table[c]:.3f} ms")
        g.close()
        pv.close()
        del pv, out, g
        torch.cuda.empty_cache()
    best = min(table, key=table.get)
    return best, table


def save_table(path, workload: str, precision: str, best, table):
    with open(path, "w") as fh:
        json.dump({"workload": workload, "precision": precision, "best_chunk": best,
                   "ms_per_launch": {str(k): v for k, v in table.items()}}, fh, indent=1)

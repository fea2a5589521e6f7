#!/usr/bin/env python3
"""Throughput benchmark of PVFinder inference (events/s) on GB300.

Workload: one batch of 1000 synthetic events per GPU (Poisson mean 5.6 PVs, ~155 tracks
per event; He-initialised weights of the 9-32x5-100 FC net and the 16/32/64/128 UNet),
the full path per step: FC + histogram, UNet, peak finding. Inputs are resident in HBM
when a step starts; L2 is flushed (512 MB write) between steps, outside the timed
events. `value` is device time (CUDA events on the launch stream, max over ranks);
`e2e` repeats the measurement through the public Python API with pinned host buffers,
including the host->device copy of the track features and offsets and the
device->host copy of the PV lists.

  python bench.py [--gpus N --steps K --warmup W] [--precision fp32|bf16|fp16|fp8]
  python bench.py --mode batch --events 50000     # one autotuned graph launch, uneven events
  python bench.py --mode serve                    # Poisson arrivals at 20k..1.5M events/s
  python bench.py --impl reference     # the FP64 CPU oracle on the host cores

The default line is the FP16 form (the paper's §5 proposal, the reduced form whose PV
lists meet the 99.9% agreement bar against the FP64 oracle); it also carries the plain
FP32 form measured on the same events with the same steps ("fp32_plain", with its own
roofline, kernels and e2e), a serving sample ("serving"), and the strict PV agreement of
the headline form with the oracle's run in the cpu_baseline leg ("pv_agreement").

With N > 1 (torchrun) every rank runs its own 1000 events (weak scaling, no
collective on the data path; events are independent).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_EVENTS = 1000
FC_MAC_PER_TRACK = 9 * 32 + 4 * 32 * 32 + 32 * 100


def conv_io(L, cin, cout, pool=False, concat=False):
    """(MAC, activation elements read, written) per event of a k5 conv layer."""
    rd = cin * (L + 4)
    wr = cout * (L + 4) + (cout * (L // 2 + 4) if pool else 0)
    return L * cout * cin * 5, rd, wr


def convT_io(L, cin, cout):
    return L * 2 * cout * cin, cin * (L + 4), cout * (2 * L + 4)


def kernel_table(form, c0=16, iv=False):
    """Work per event of each kernel family: (tensor-core MAC, CUDA-core MAC, activation
    bytes read + written), for UNet base width c0 (levels c0, 2 c0, 4 c0, 8 c0); iv: the
    per-interval layout (40 sequences of 104 bins per event instead of one of 4000). The
    FC's MACs depend on the track count and are added by the caller (front kernel). The
    activation bytes are those the implementation stores between kernels, not work the
    method requires (its own bytes are the input tracks and the PV lists)."""
    es = {"fp32": 4, "bf16": 2, "fp16": 2, "fp8": 1}[form]
    tc = form != "fp32"
    c1, c2, c3, c4 = c0, 2 * c0, 4 * c0, 8 * c0
    L0, q = (104, 40) if iv else (4000, 1)             # sequence length, sequences per event
    L1, L2, L3 = L0 // 2, L0 // 4, L0 // 8

    def scaled(mrw):
        return tuple(q * x for x in mrw)

    def entry(mac, nbytes, alu_mac=0):
        return (mac, alu_mac, nbytes) if tc else (0, mac + alu_mac, nbytes)

    t = {}
    e1 = q * (c1 * (L0 + 4) + c1 * (L1 + 4))            # e1 and p1 written by the front kernel
    t["front"] = (0, q * L0 * c1 * 5, e1 * es)          # enc1 on CUDA cores; + the FC, + 36 B per track
    m, r, w = scaled(conv_io(L1, c1, c2, pool=True)); t["enc2"] = entry(m, (r + w) * es)
    m, r, w = scaled(conv_io(L2, c2, c3, pool=True)); t["enc3"] = entry(m, (r + w) * es)
    if form == "fp32":
        m, r, w = scaled(conv_io(L3, c3, c4)); t["enc4"] = entry(m, (r + w) * es)
        m, r, w = scaled(convT_io(L3, c4, c3)); t["up3"] = entry(m, (r + w) * es)
        m, r, w = scaled(conv_io(L2, 2 * c3, c3)); t["dec3"] = entry(m, (r + w) * es)
        m, r, w = scaled(convT_io(L2, c3, c2)); t["up2"] = entry(m, (r + w) * es)
        m, r, w = scaled(conv_io(L1, 2 * c2, c2)); t["dec2"] = entry(m, (r + w) * es)
        m, r, w = scaled(convT_io(L1, c2, c1)); t["up1"] = entry(m, (r + w) * es)
        m, r, w = scaled(conv_io(L0, 2 * c1, c1)); t["dec1"] = entry(m, (r + w) * es)
        t["tail"] = (0, 4000 * c1 * 5, q * c1 * (L0 + 4) * es + 16000)
    elif c0 == 32 and not iv:
        # the wide network: enc4 and dec3 split over CTAs store e4 and d3; up3 and up2 run
        # as ConvT kernels of their own
        m, r, w = conv_io(L3, c3, c4); t["enc4"] = entry(m, (r + w) * es)
        m, r, w = convT_io(L3, c4, c3); t["up3"] = entry(m, (r + w) * es)
        m, r, w = conv_io(L2, 2 * c3, c3); t["dec3"] = entry(m, (r + w) * es)
        m, r, w = convT_io(L2, c3, c2); t["up2"] = entry(m, (r + w) * es)
        m1, r1, _ = conv_io(L1, 2 * c2, c2); m2, _, w2 = convT_io(L1, c2, c1)
        t["dec2_up1"] = entry(m1 + m2, (r1 + w2) * es)
        m1, r1, _ = conv_io(L0, 2 * c1, c1)
        t["dec1_final"] = entry(m1, r1 * es + 16000, alu_mac=L0 * c1 * 5)
        t["tail"] = (0, 0, 16000)
    else:
        m1, r1, _ = scaled(conv_io(L3, c3, c4)); m2, _, w2 = scaled(convT_io(L3, c4, c3))
        t["enc4_up3"] = entry(m1 + m2, (r1 + w2) * es)
        m1, r1, _ = scaled(conv_io(L2, 2 * c3, c3)); m2, _, w2 = scaled(convT_io(L2, c3, c2))
        t["dec3_up2"] = entry(m1 + m2, (r1 + w2) * es)
        m1, r1, _ = scaled(conv_io(L1, 2 * c2, c2)); m2, _, w2 = scaled(convT_io(L1, c2, c1))
        t["dec2_up1"] = entry(m1 + m2, (r1 + w2) * es)
        m1, r1, _ = scaled(conv_io(L0, 2 * c1, c1))
        # the final conv (fp32, CUDA cores) at the 4000 bins that get logits
        t["dec1_final"] = entry(m1, r1 * es + 16000, alu_mac=4000 * c1 * 5)
        t["tail"] = (0, 0, 16000)
    return t


def peak_rates(peaks, form):
    """Peak rates the fractions are taken against: tensor FLOP/s for the form's operand
    type (measured bf16 burst; fp16 = bf16; e4m3 = 2 x bf16, the nominal ratio), fp32
    CUDA-core FLOP/s and SFU operations/s derived from unit counts and the maximum SM
    clock (152 SMs x 128 fp32 lanes x 2; 152 SMs x 16 SFU lanes), HBM bytes/s (measured)."""
    clk = peaks.get("sm_max_mhz", 2070.0) * 1e6
    return {"tensor": peaks["bf16_tflops"] * 1e12 * (2.0 if form == "fp8" else 1.0),
            "alu": 152 * 128 * 2 * clk, "sfu": 152 * 16 * clk, "hbm": peaks["hbm_gbs"] * 1e9}


def roofline_of(name, launches, tot_ms, form, events_per_launch, tracks_per_launch, peaks,
                fc_evals=None, c0=16, iv=False):
    """Roofline of one kernel family from the method's work per launch (MACs of the layers
    it computes) over its measured launch duration. The bound is the compute unit that
    does the kernel's arithmetic: the tensor pipe for the UNet convolutions of the
    tensor-core forms, the fp32 CUDA cores for the float32 form. `hbm_frac` is the
    activation bytes the implementation moves (not required by the method) over the
    measured HBM bandwidth. The front kernel runs the FC on the tensor pipe, softplus on
    the SFU and enc1 on CUDA cores, and is reported against each; its bound is
    "latency" when none of them is near its peak. fc_evals: FC evaluations per launch
    (tracks plus second slices of boundary tracks)."""
    tc_mac, alu_mac, bytes_ev = kernel_table(form, c0, iv)[name]
    sec = tot_ms / max(launches, 1) / 1000.0
    pk = peak_rates(peaks, form)
    nbytes = bytes_ev * events_per_launch
    if name == "front":
        fe = tracks_per_launch if fc_evals is None else fc_evals
        nbytes += 36.0 * tracks_per_launch
        fc_flops = 2.0 * FC_MAC_PER_TRACK * fe
        alu_flops = 2.0 * alu_mac * events_per_launch + (0 if form != "fp32" else fc_flops)
        fracs = {"alu": alu_flops / sec / pk["alu"],
                 "sfu": 200.0 * fe / sec / pk["sfu"],          # softplus: exp2 + log2 per output
                 "hbm": nbytes / sec / pk["hbm"]}
        if form != "fp32":
            fracs["tensor"] = fc_flops / sec / pk["tensor"]
        top = max(fracs, key=fracs.get)
        return {"bound": top if fracs[top] >= 0.5 else "latency", "frac": fracs[top],
                "unit_fracs": fracs, "achieved": fracs[top] * pk[top] / (1e9 if top == "hbm" else 1e12),
                "peak": pk[top] / (1e9 if top == "hbm" else 1e12),
                "unit": "GB/s" if top == "hbm" else ("TOP/s" if top == "sfu" else "TFLOP/s"),
                "hbm_frac": nbytes / sec / pk["hbm"], "activation_bytes": nbytes}
    if tc_mac == 0 and alu_mac == 0:              # the tail of the tensor-core forms: reads logits
        return {"bound": "hbm", "achieved": nbytes / sec / 1e9, "peak": pk["hbm"] / 1e9,
                "unit": "GB/s", "frac": nbytes / sec / pk["hbm"], "hbm_frac": nbytes / sec / pk["hbm"],
                "activation_bytes": nbytes}
    kind, mac = ("tensor", tc_mac) if tc_mac else ("alu", alu_mac)
    flops = 2.0 * mac * events_per_launch
    return {"bound": kind, "achieved": flops / sec / 1e12, "peak": pk[kind] / 1e12, "unit": "TFLOP/s",
            "frac": flops / sec / pk[kind], "algorithmic_flops": flops,
            "hbm_frac": nbytes / sec / pk["hbm"], "activation_bytes": nbytes}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the kernels that
# can dominate a step, from ncu captures of the kernels as built (profiles/ gives the
# commands). Keyed by (form, kernel, events per launch); the value is (bytes, source). A
# kernel changed since its capture has no entry and reports null.
NCU_TRAFFIC = {
    ("fp16", "dec3_up2", 1000): ((257.183744e6 + 90.259456e6),
                                 "ncu --set full of one 1000-event launch (profiles/dec3_up2_fp16_1000ev.md)"),
}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def rank_workload_seed(rank: int) -> int:
    """Each rank draws its own events (weak scaling): no event is shared between ranks."""
    return 1000 + rank


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The slowest rank's time: all_reduce(MAX) of one float (the only collective, outside
    the timed region)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(events_per_rank: int, world: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput: all ranks' events over the slowest rank's device time."""
    return events_per_rank * world * steps / (max_ms / 1000.0)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms around the timed region:
    the sampler is running (its first sample taken) before the warm-up steps start, and the
    caller keeps the GPU busy with the same steps for a while after the timed ones, so the
    samples come from the GPU under this load even when the timed steps last a few ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200",
                                          "-i", str(self.gpu)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def wait_first(self, timeout_s=5.0):
        """Returns once nvidia-smi has written its first sample (or after timeout_s)."""
        t0 = time.perf_counter()
        while self.proc and time.perf_counter() - t0 < timeout_s:
            self.fh.flush()
            if os.path.getsize(self.path) > 0:
                return
            time.sleep(0.02)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "window": "nvidia-smi every 200 ms from before the warm-up steps "
                                              "through the timed steps and 0.6 s of further steps"}


def oracle_cpu_baseline(weights, batch, target_s=10.0, max_events=None, **variant):
    """Times the FP64 oracle (as it stands) on a bounded sample of the workload, all cores.
    variant: the oracle's edge_mm / per_interval, matching the GPU run. Returns the
    baseline and the oracle's results on the sample (its PV lists and logits)."""
    import oracle
    cores = os.cpu_count() or 1
    n0 = min(batch.n_events, cores)
    sub = batch.subset(0, n0)
    t0 = time.perf_counter()
    oracle.infer(weights, sub.features, sub.offsets, max_pv=672, nthreads=cores, **variant)
    dt0 = time.perf_counter() - t0
    n = int(min(batch.n_events, max(n0, n0 * target_s / max(dt0, 1e-3))))
    if max_events:
        n = min(n, max_events)
    n = max(n0, n // cores * cores)
    sub = batch.subset(0, n)
    t0 = time.perf_counter()
    ref = oracle.infer(weights, sub.features, sub.offsets, max_pv=672, want_logit=True,
                       nthreads=cores, **variant)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "events/s", "cores": min(cores, n), "kind": "oracle",
            "sample": f"first {n} of the {batch.n_events}-event workload, FP64 C oracle, "
                      f"one event per thread, {dt:.1f} s wall"}, ref


def oracle_variant(args):
    """The oracle's options for the workload variant the GPU run uses."""
    return {"edge_mm": args.boundary_mm, "per_interval": args.per_interval}


def run_reference(args, weights, batch, rank, world):
    """--impl reference: the FP64 CPU oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    cores = os.cpu_count() or 1
    per_step = cores
    n = batch.n_events
    times = []
    for step in range(args.warmup + args.steps):
        a = (step * per_step) % n
        b = min(n, a + per_step)
        sub = batch.subset(a, b)
        t0 = time.perf_counter()
        oracle.infer(weights, sub.features, sub.offsets, max_pv=256, nthreads=cores,
                     **oracle_variant(args))
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append((b - a, dt))
    ev = sum(t[0] for t in times)
    sec = sum(t[1] for t in times)
    value = ev / sec
    line = {
        "impl": "reference", "metric": "events/s", "value": value, "unit": "events/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * sec / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, "f64"),
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} events per step (one per core), rotating through "
                                   f"the {n}-event workload"},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def fc_evaluations(batch, edge):
    """FC evaluations of a batch: one per track, plus one per boundary track (a track
    whose slice-relative z is below `edge` mm, above slice 0, or at least 10 - edge,
    below slice 39), decided in float32 as the kernels do."""
    n = int(np.sum(np.diff(batch.offsets)))
    if edge <= 0:
        return n
    z = batch.features[2].astype(np.float32)
    with np.errstate(invalid="ignore"):
        s = np.floor((z + np.float32(100.0)) / np.float32(10.0))
    ok = np.isfinite(s) & (s >= 0) & (s < 40)
    s = np.where(ok, s, 0).astype(np.float32)
    zr = z - (np.float32(-100.0) + np.float32(10.0) * s)
    lo = ok & (s > 0) & (zr < np.float32(edge))
    hi = ok & (s < 39) & (zr >= np.float32(10.0) - np.float32(edge))
    return n + int(lo.sum() + hi.sum())


def workload_config(args, dtype):
    return {"workload": f"PVFinder inference, {args.events} synthetic events per GPU "
                        f"(~155 tracks/event, Poisson 5.6 PVs), 4000-bin histogram, "
                        f"{'/'.join(str(args.unet_width * k) for k in (1, 2, 4, 8))} UNet, {dtype}",
            "events_per_gpu": args.events, "bins": 4000, "max_pv_per_event": args.max_pv,
            "l2": f"flushed between steps ({args.flush_mb} MB write)" if args.flush_mb >= 256
                  else "not flushed (profiling run)", "form": args.precision,
            "boundary_mm": args.boundary_mm, "unet_width": args.unet_width,
            "per_interval": args.per_interval}


def make_finder(args, weights, precision, events, **kw):
    """PVFinder for `precision`; FP8 scales come from a calibration pass (512 seeded
    events, seed 1, through a BF16 handle) outside any timed region."""
    import torch
    import synth
    from paper_2602_19959_gb300 import PVFinder
    scales = None
    if precision == "fp8":
        cal = synth.generate_standard(512, 1)
        pcal = PVFinder(weights, precision="bf16", max_events=512, max_pv_per_event=8)
        scales = pcal.calibrate(torch.from_numpy(cal.features).cuda(),
                                torch.from_numpy(cal.offsets).cuda())
        pcal.close()
    return PVFinder(weights, precision=precision, max_events=events, fp8_act_scales=scales,
                    boundary_mm=args.boundary_mm, per_interval=args.per_interval, **kw)


def time_steps(pv, step, flush, steps, world, profile):
    """K steps, each bracketed by CUDA events on the launch stream; L2 flushed between
    steps outside the events; barrier + synchronize on both sides."""
    import torch
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    prof = {}
    pv.profile_enable(profile)
    barrier(world)
    w0 = time.perf_counter()
    for i in range(steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        if profile:
            for k, (n, ms) in pv.profile_read().items():
                a = prof.setdefault(k, [0, 0.0])
                a[0] += n
                a[1] += ms
    barrier(world)
    wall = time.perf_counter() - w0
    pv.profile_enable(False)
    return sum(a.elapsed_time(b) for a, b in ev), wall, prof


def time_e2e_pipelined(pv, feats_h, offs_h, out_shapes, steps, world):
    """End-to-end steps through the public API with host buffers, double-buffered the way a
    streaming caller runs it: every step copies its inputs host->device from pinned memory
    and reads its PV lists back while the compute stream runs the neighbouring steps
    (inputs and outputs on two copy streams, so a step's input copy never queues behind the
    previous step's readback). Returns the total milliseconds of `steps` steps (events on
    the compute stream, which the copy streams join at both ends)."""
    import torch
    comp = torch.cuda.current_stream()
    cp_in, cp_out = torch.cuda.Stream(), torch.cuda.Stream()
    dev_in = [(torch.empty_like(feats_h, device="cuda"), torch.empty_like(offs_h, device="cuda"))
              for _ in range(2)]
    dev_out = [pv.alloc_outputs(out_shapes) for _ in range(2)]
    host_out = [(torch.empty(dev_out[0][0].shape, dtype=dev_out[0][0].dtype).pin_memory(),
                 torch.empty(dev_out[0][1].shape, dtype=dev_out[0][1].dtype).pin_memory())
                for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_comp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    t0.record(comp)
    cp_in.wait_stream(comp)
    cp_out.wait_stream(comp)
    for i in range(steps):
        j = i & 1
        with torch.cuda.stream(cp_in):
            if i >= 2:
                cp_in.wait_event(ev_comp[j])           # step i - 2 no longer reads these inputs
            dev_in[j][0].copy_(feats_h, non_blocking=True)
            dev_in[j][1].copy_(offs_h, non_blocking=True)
            ev_in[j].record(cp_in)
        comp.wait_event(ev_in[j])
        if i >= 2:
            comp.wait_event(ev_out[j])                 # step i - 2's results are read back
        pv.infer(dev_in[j][0], dev_in[j][1], out=dev_out[j], stream=comp)
        ev_comp[j].record(comp)
        with torch.cuda.stream(cp_out):
            cp_out.wait_event(ev_comp[j])
            host_out[j][0].copy_(dev_out[j][0], non_blocking=True)
            host_out[j][1].copy_(dev_out[j][1], non_blocking=True)
            ev_out[j].record(cp_out)
    comp.wait_stream(cp_in)
    comp.wait_stream(cp_out)
    t1.record(comp)
    torch.cuda.synchronize()
    barrier(world)
    return t0.elapsed_time(t1)


def barrier(world):
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()


def serve_sample(pv, store, rate, seconds, seed, max_batch, max_inflight, copy=False, lead_us=0.0):
    """Poisson arrivals at `rate` events/s for `seconds` through pvf_serve_replay; latency is
    arrival -> the host seeing its batch complete (results readable on the host)."""
    rng = np.random.default_rng(seed)
    n = int(rate * seconds)
    arrivals = np.cumsum(rng.exponential(1e9 / rate, n)).astype(np.int64)
    req = (np.arange(n) % store.n_events).astype(np.int32)
    t0 = time.perf_counter()
    done, cnt, batches, _ = pv.serve_replay(store, arrivals, req, max_batch=max_batch,
                                            max_inflight=max_inflight, copy=copy,
                                            launch_lead_us=lead_us)
    wall = time.perf_counter() - t0
    lat = (done - arrivals) / 1000.0
    return {"rate_offered": rate, "events": n, "seconds": seconds,
            "events_per_s": n / ((done.max() - arrivals.min()) / 1e9),
            "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
            "p999_us": float(np.percentile(lat, 99.9)), "max_us": float(lat.max()),
            "batches": batches, "mean_batch": n / max(batches, 1), "wall_s": wall,
            "form": "copy" if copy else "gather (zero-copy)", "launch_lead_us": lead_us,
            "max_batch": max_batch, "max_inflight": max_inflight,
            "under_400us_p99": bool(np.percentile(lat, 99) < 400.0)}


def measure_form(args, weights, batch, precision, feats, offs, feats_h, offs_h, flush, world, local,
                 clocks_too=False):
    """One form of the path on the rank's batch: device-timed steps, the same steps with
    per-kernel events (breakdown and roofline), and end-to-end steps through the public API
    on pinned host buffers. Returns (line fields, the finder, its device outputs)."""
    import torch
    dtype = {"fp32": "f32", "bf16": "bf16", "fp16": "f16", "fp8": "e4m3"}[precision]
    pv = make_finder(args, weights, precision, args.events, max_pv_per_event=args.max_pv)
    z, c = pv.alloc_outputs(args.events)

    def step_device():
        pv.infer(feats, offs, out=(z, c))

    sampler = ClockSampler(local) if clocks_too else None
    if sampler:
        sampler.start()
        sampler.wait_first()
    for _ in range(args.warmup):
        flush.fill_(1)
        step_device()
    torch.cuda.synchronize()
    status = pv.device_status()

    # whole steps only (per-kernel events between launches would also stop the kernels'
    # dependent launches from overlapping one kernel's tail with the next one's prologue);
    # then the same steps again with per-kernel events for the breakdown
    dev_ms, wall, _ = time_steps(pv, step_device, flush, args.steps, world, False)
    clocks = None
    if sampler:
        t_busy = time.perf_counter()
        while time.perf_counter() - t_busy < 0.6:     # the same load, untimed, for the sampler
            flush.fill_(1)
            step_device()
            torch.cuda.synchronize()
        clocks = sampler.stop()
    prof_ms, _, prof = time_steps(pv, step_device, flush, args.steps, world, True)
    e2e_ms = time_e2e_pipelined(pv, feats_h, offs_h, args.events, args.steps, world)

    dev_ms = max_over_ranks(dev_ms, world, "cuda")
    e2e_ms = max_over_ranks(e2e_ms, world, "cuda")
    value = aggregate_value(args.events, world, args.steps, dev_ms)
    e2e_value = aggregate_value(args.events, world, args.steps, e2e_ms)

    # dominant kernel and its roofline (the method's work / live launch duration)
    peaks, peak_src = load_peaks()
    valid_tracks = int(np.sum(np.diff(batch.offsets)))
    fc_evals = fc_evaluations(batch, args.boundary_mm)
    kernels = {}
    total_ms = max(sum(v[1] for v in prof.values()), 1e-9)
    for k, (n, ms) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
        rf = roofline_of(k, n, ms, precision, args.events, valid_tracks, peaks, fc_evals,
                         args.unet_width, args.per_interval)
        kernels[k] = {"launches": n, "avg_us": 1000.0 * ms / max(n, 1), "share": ms / total_ms,
                      "bound": rf["bound"], "frac": rf["frac"], "hbm_frac": rf["hbm_frac"]}
        if "unit_fracs" in rf:
            kernels[k]["unit_fracs"] = rf["unit_fracs"]
    name, (launches, tot_ms) = max(prof.items(), key=lambda kv: kv[1][1])
    roof = roofline_of(name, launches, tot_ms, precision, args.events, valid_tracks, peaks, fc_evals,
                       args.unet_width, args.per_interval)
    traffic = NCU_TRAFFIC.get((precision, name, args.events))
    roof.update({"kernel": name, "traffic": traffic[0] if traffic else None,
                 "traffic_source": traffic[1] if traffic else "no ncu capture of this kernel as built",
                 "peak_source": f"{peak_src} (MEASURED_PEAKS.json: bf16_tflops burst, hbm_gbs; fp16 = "
                                "bf16; e4m3 = 2 x bf16; fp32 ALU = 152 SM x 128 lanes x 2 x sm_max_mhz)"})
    h2d = batch.features.nbytes + batch.offsets.nbytes
    d2h = z.numel() * 4 + c.numel() * 4
    out = {
        "value": value, "ms_per_step": dev_ms / args.steps,
        "ms_per_step_with_kernel_events": prof_ms / args.steps, "dtype": dtype, "form": precision,
        "e2e": {"value": e2e_value, "unit": "events/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "how": "pvf_infer per step on pinned host inputs and outputs, the copies of "
                       "step i+1 / i-1 overlapping step i's compute (two buffer sets, an "
                       "input and an output copy stream)"},
        "roofline": roof, "kernels": kernels, "gpu_launches": int(sum(n for n, _ in prof.values())),
        "device_status": status, "wall_s_timed": wall,
    }
    if clocks_too:
        out["clocks"] = clocks
    return out, pv, (z, c)


def gpu_logits(pv, feats, offs, n):
    """PV lists and logits of the first n events of the batch (outside any timed region),
    for the agreement with the oracle's run."""
    import torch
    logit = torch.zeros((n, 4000), dtype=torch.float32, device="cuda")
    z, c = pv.alloc_outputs(n)
    pv.infer(feats, offs[:n + 1], n_events=n, out=(z, c), logit=logit)
    torch.cuda.synchronize()
    return z.cpu().numpy(), c.cpu().numpy(), logit.cpu().numpy()


def run_step(args, weights, batch, rank, world, local):
    import torch
    from paper_2602_19959_gb300 import build
    from paper_2602_19959_gb300.agreement import pv_agreement
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build()
    barrier(world)

    feats_h = torch.from_numpy(batch.features).pin_memory()
    offs_h = torch.from_numpy(batch.offsets).pin_memory()
    feats = feats_h.cuda()
    offs = offs_h.cuda()
    flush = torch.empty(max(args.flush_mb, 1) * 1024 * 1024, dtype=torch.uint8, device="cuda")

    head, pv, _ = measure_form(args, weights, batch, args.precision, feats, offs, feats_h, offs_h,
                               flush, world, local, clocks_too=True)
    line = {
        "metric": "events/s", "value": head["value"], "unit": "events/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": head["dtype"],
        "data": "synthetic", "config": workload_config(args, head["dtype"]),
    }
    line.update({k: v for k, v in head.items() if k not in line and k not in ("value",)})
    agree_pv = pv
    if args.compare and args.precision != "fp32":
        # the plain FP32 GPU form on the same events, same steps and the same measurements
        p32_line, p32, _ = measure_form(args, weights, batch, "fp32", feats, offs, feats_h, offs_h,
                                        flush, world, local)
        p32_line["speedup_of_headline"] = head["value"] / p32_line["value"]
        line["fp32_plain"] = p32_line
        p32.close()
        del p32
    if args.serve_seconds > 0 and world == 1:
        import synth
        store = synth.generate_uneven(4096, 55)
        ps = make_finder(args, weights, args.precision, args.serve_batch,
                         max_pv_per_event=args.max_pv)
        line["serving"] = serve_sample(ps, store, args.serve_rate, args.serve_seconds, 7,
                                       args.serve_batch, args.serve_inflight, copy=args.serve_copy,
                                       lead_us=args.serve_lead_us)
        line["serving"]["workload"] = "uneven events (N_PV ~ U{1..12}, heavy-tailed background)"
        ps.close()
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        cb, ref = oracle_cpu_baseline(weights, batch, **oracle_variant(args))
        line["cpu_baseline"] = cb
        n = len(ref["pv_count"])
        gz, gc, gl = gpu_logits(agree_pv, feats, offs, n)
        a = pv_agreement(ref["pv_z"], ref["pv_count"], gz, gc, ref["logit"], gl)
        line["pv_agreement"] = {
            "form": args.precision, "events": n, "strict": a["strict"], "exempt": a["exempt"],
            "matched": a["matched"], "total": a["total"], "max_dz_mm": a["max_dz"],
            "source": "the FP64 oracle's run of the cpu_baseline leg (same events); exempt: "
                      "disagreements the measured per-bin logit differences can flip"}
    pv.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batch(args, weights):
    """Config 4: uneven events (N_PV ~ U{1..12}, heavy-tailed background) as one persistent,
    graph-captured launch. The autotuner's table for this workload and form is read from
    paper_2602_19959_gb300/tuned/ (or written there with --retune); the line reports the
    launch with the tuned schedule and with the defaults."""
    import torch
    import synth
    from paper_2602_19959_gb300 import build
    from paper_2602_19959_gb300 import autotune as T
    from paper_2602_19959_gb300.pvf import PVFinder
    build()
    b = synth.generate_uneven(args.events, 4)
    workload = f"uneven{args.events}"
    path = args.tune_out or T.table_path(args.precision, workload)
    log = (lambda m: print(m, file=sys.stderr, flush=True))
    if args.retune or not os.path.exists(path):
        best, trials = T.tune(weights, b, args.precision, chunk_candidates=(0, 12500, 5000, 2000),
                              repeats=min(args.steps, 3), max_pv=args.max_pv, log=log)
        T.save_table(path, workload, args.precision, best, trials, trials[0]["ms"])
    chunk, sched = T.load_schedule(path)
    feats = torch.from_numpy(b.features).cuda()
    offs = torch.from_numpy(b.offsets).cuda()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    res = {}
    for name, (ck, sc) in (("tuned", (chunk, sched)), ("default", (0, None))):
        pv = PVFinder(weights, precision=args.precision, max_events=args.events, chunk_events=ck,
                      max_pv_per_event=args.max_pv, schedule=sc)
        res[name] = T._time_graph(pv, feats, offs, max(args.steps, 3), max(args.warmup, 1), flush)
        res[name + "_pool_bytes"] = pv.pool_bytes
        pv.close()
        del pv
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "events/s (one graph launch)", "value": args.events / (res["tuned"] / 1000.0),
                      "unit": "events/s", "workload": f"{args.events} uneven events (N_PV ~ U{{1..12}}, "
                      f"Pareto(2, 5) background capped at 400), one graph launch",
                      "dtype": args.precision, "ms_per_launch": res["tuned"],
                      "default_schedule_ms": res["default"],
                      "default_schedule_events_per_s": args.events / (res["default"] / 1000.0),
                      "schedule": {"chunk_events": chunk or args.events, **sched},
                      "pool_bytes": res["tuned_pool_bytes"], "tune_table": os.path.relpath(path, ROOT),
                      "l2": "flushed between launches (512 MB write)", "timing": "min over launches"}),
          flush=True)


def run_serve(args, weights):
    """Serving: Poisson arrivals at each offered rate for serve_seconds_full, through the
    continuous-batching loop; one JSON line per rate."""
    import synth
    from paper_2602_19959_gb300 import build
    build()
    store = synth.generate_uneven(args.serve_store, 55)
    pv = make_finder(args, weights, args.precision, args.serve_batch, max_pv_per_event=args.max_pv)
    for rate in args.rates:
        r = serve_sample(pv, store, rate, args.serve_seconds_full, 100 + int(rate // 1000),
                         args.serve_batch, args.serve_inflight, copy=args.serve_copy,
                         lead_us=args.serve_lead_us)
        r.update({"metric": "serving latency", "dtype": args.precision,
                  "workload": f"Poisson arrivals over {args.serve_store} stored uneven events (cycled)",
                  "pool_bytes": pv.pool_bytes})
        print(json.dumps(r), flush=True)
    pv.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["step", "batch", "serve"], default="step")
    ap.add_argument("--precision", default="fp16", choices=["fp32", "bf16", "fp16", "fp8"])
    ap.add_argument("--events", type=int, default=N_EVENTS)
    ap.add_argument("--max-pv", type=int, default=672)
    ap.add_argument("--unet-width", type=int, default=16, choices=[16, 32],
                    help="UNet base width (32: the wide variant)")
    ap.add_argument("--per-interval", action="store_true",
                    help="each interval runs the UNet as its own 104-bin sequence")
    ap.add_argument("--boundary-mm", type=float, default=0.0,
                    help="boundary tracks fill a second slice within this width (0: none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip the plain FP32 comparison run")
    ap.add_argument("--flush-mb", type=int, default=512,
                    help="L2 flush buffer written between steps (0: none, for small profiling runs)")
    ap.add_argument("--serve-seconds", type=float, default=2.0,
                    help="serving sample folded into the step line (0: none)")
    ap.add_argument("--serve-rate", type=float, default=870000.0,
                    help="offered rate of that sample (5x the plain FP32 form's throughput)")
    ap.add_argument("--serve-batch", type=int, default=512)
    ap.add_argument("--serve-inflight", type=int, default=1,
                    help="batches enqueued at once (1 measured lowest p99: the next batch takes "
                         "every request that arrives while one runs)")
    ap.add_argument("--serve-copy", action="store_true",
                    help="serving: the copy form (device slots, per-bucket graphs)")
    ap.add_argument("--serve-lead-us", type=float, default=0.0,
                    help="serving: admit the next batch only when the running one is predicted "
                         "to end within this many us (0: whenever a slot is free)")
    ap.add_argument("--serve-seconds-full", type=float, default=10.0)
    ap.add_argument("--serve-store", type=int, default=200000,
                    help="serve mode: distinct stored events the requests cycle through")
    ap.add_argument("--retune", action="store_true",
                    help="batch mode: run the autotuner even if its table exists")
    ap.add_argument("--tune-out", default=None, help="batch mode: where to write / read the table")
    ap.add_argument("--rates", type=float, nargs="+",
                    default=[20000, 60000, 120000, 200000, 500000, 870000, 1200000, 1500000])
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    import synth
    rank, world, local = dist_env()
    if args.per_interval and args.unet_width != 16:
        ap.error("--per-interval exists at width 16 only")
    weights = synth.he_weights(0, c0=args.unet_width)
    if args.impl == "reference":
        batch = synth.generate_standard(args.events, rank_workload_seed(rank))
        run_reference(args, weights, batch, rank, world)
        return
    import torch
    torch.cuda.set_device(local)
    if args.mode == "batch":
        run_batch(args, weights)
        return
    if args.mode == "serve":
        run_serve(args, weights)
        return
    batch = synth.generate_standard(args.events, rank_workload_seed(rank))
    run_step(args, weights, batch, rank, world, local)


if __name__ == "__main__":
    main()

"""Batching and serving through the C ABI: the graph-captured launch and the
continuous-batching request loop. Each result must be the same alone and in the mix:
the path is batch-invariant bit for bit, so the comparison is exact."""

import numpy as np
import pytest

import synth
from tests.helpers import to_cuda

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def PVFinder():
    from paper_2602_19959_gb300 import build, PVFinder
    build()
    return PVFinder


@pytest.fixture(scope="module")
def weights():
    return synth.he_weights(0)


def alone(pv, batch, max_pv):
    """Each event run by itself: (counts [n], z [n, max_pv])."""
    n = batch.n_events
    cnt = np.zeros(n, np.int32)
    z = np.zeros((n, max_pv), np.float32)
    for e in range(n):
        sub = batch.subset(e, e + 1)
        zz, cc = pv.infer(*to_cuda(sub))
        torch.cuda.synchronize()
        cnt[e] = cc.cpu().numpy()[0]
        z[e] = zz.cpu().numpy()[0]
    return cnt, z


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_graph_launch_matches_infer_and_follows_new_inputs(PVFinder, weights, precision):
    b1 = synth.generate_uneven(48, 11)
    b2 = synth.generate_uneven(48, 12)
    cap = int(max(b1.n_tracks, b2.n_tracks))
    pv = PVFinder(weights, precision=precision, max_events=48, chunk_events=16, max_pv_per_event=96)
    feats = torch.zeros((9, cap), dtype=torch.float32, device="cuda")
    offs = torch.zeros(49, dtype=torch.int32, device="cuda")
    out = pv.alloc_outputs(48)
    g = pv.capture_graph(feats, offs, out)
    for b in (b1, b2):
        feats.zero_()
        feats[:, :b.n_tracks] = torch.from_numpy(b.features).cuda()
        offs.copy_(torch.from_numpy(b.offsets).cuda())
        g.launch()
        torch.cuda.synchronize()
        gz, gc = out[0].cpu().numpy().copy(), out[1].cpu().numpy().copy()
        zz, cc = pv.infer(feats, offs)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(gc, cc.cpu().numpy())
        zz = zz.cpu().numpy()
        for e in range(48):            # slots past an event's count are left untouched
            k = min(int(gc[e]), 96)
            np.testing.assert_array_equal(gz[e, :k], zz[e, :k])
    g.close()


@pytest.mark.parametrize("precision,boundary_mm", [("fp32", 0.0), ("bf16", 0.0), ("fp16", 0.0), ("fp16", 0.5)])
def test_launch_schedule_changes_nothing_but_the_grids(PVFinder, weights, precision, boundary_mm):
    """Every kernel walks its work whatever its grid, and no sum depends on which CTA takes
    which event or tile: results are bit for bit the same under any launch schedule,
    including both shapes of the front (256-thread CTAs at 1-2 per SM, 128-thread CTAs at
    3-4), which split every bin's sum at the same multiples of 128 sorted tracks."""
    b = synth.generate_uneven(96, 17)
    feats, offs = to_cuda(b)
    outs = []
    for sched in (None, {"front": 1, "enc2": 2, "enc3": 1, "dec2_up1": 1, "dec1_final": 2, "tail": 1},
                  {"front": 2, "enc2": 99, "dec1_final": 3, "tail": 4}, {"front": 3}, {"front": 4}):
        pv = PVFinder(weights, precision=precision, max_events=96, max_pv_per_event=96, schedule=sched,
                      boundary_mm=boundary_mm)
        hist = torch.zeros((96, 4000), device="cuda")
        logit = torch.zeros((96, 4000), device="cuda")
        z, c = pv.infer(feats, offs, hist=hist, logit=logit)
        torch.cuda.synchronize()
        outs.append((hist.cpu().numpy(), logit.cpu().numpy(), c.cpu().numpy()))
        pv.close()
    for o in outs[1:]:
        for x, y in zip(o, outs[0]):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("precision", ["bf16", "fp16", "fp8"])
def test_dynamic_graph_follows_the_device_side_count(PVFinder, weights, precision, request):
    """One graph captured for 48 events, launched with 48, 17, 1, 0 and 30 events as its
    device-side count: each launch gives pvf_infer's results on the first n events and
    writes no count past them."""
    kw = {}
    if precision == "fp8":
        cal = synth.generate_standard(512, 1)
        pc = PVFinder(weights, precision="bf16", max_events=512, max_pv_per_event=8)
        kw["fp8_act_scales"] = pc.calibrate(*to_cuda(cal))
        pc.close()
    b = synth.generate_uneven(48, 13)
    pv = PVFinder(weights, precision=precision, max_events=48, chunk_events=16, max_pv_per_event=96, **kw)
    feats, offs = to_cuda(b)
    n_dev = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = pv.alloc_outputs(48)
    g = pv.capture_graph_dynamic(feats, offs, n_dev, out)
    zz, cc = pv.infer(feats, offs)
    torch.cuda.synchronize()
    ref_c, ref_z = cc.cpu().numpy(), zz.cpu().numpy()
    for n in (48, 17, 1, 0, 30):
        out[1].fill_(-7)
        n_dev.fill_(n)
        g.launch()
        torch.cuda.synchronize()
        gc, gz = out[1].cpu().numpy(), out[0].cpu().numpy()
        np.testing.assert_array_equal(gc[:n], ref_c[:n])
        assert np.all(gc[n:] == -7)
        for e in range(n):
            k = min(int(gc[e]), 96)
            np.testing.assert_array_equal(gz[e, :k], ref_z[e, :k])
    from paper_2602_19959_gb300.pvf import PVF_WARN_TRUNCATED
    assert pv.device_status() in (0, PVF_WARN_TRUNCATED)        # 96 slots: some lists truncated
    g.close()


def test_dynamic_graph_is_refused_by_the_float32_form(PVFinder, weights):
    from paper_2602_19959_gb300.pvf import PvfError, PVF_ERR_UNSUPPORTED
    pv = PVFinder(weights, precision="fp32", max_events=8)
    b = synth.generate_uneven(8, 2)
    feats, offs = to_cuda(b)
    n_dev = torch.full((1,), 8, dtype=torch.int32, device="cuda")
    with pytest.raises(PvfError) as ei:
        pv.capture_graph_dynamic(feats, offs, n_dev, pv.alloc_outputs(8))
    assert ei.value.code == PVF_ERR_UNSUPPORTED


@pytest.mark.parametrize("graphs,copy,max_batch,inflight,precision,lead",
                         [(True, False, 32, 3, "bf16", 0.0), (True, False, 24, 1, "fp16", 0.0),
                          (True, False, 32, 2, "fp16", 20.0),
                          (True, True, 32, 3, "bf16", 0.0), (True, True, 24, 1, "bf16", 0.0),
                          (False, True, 32, 2, "bf16", 0.0), (True, False, 32, 2, "fp8", 0.0),
                          (True, True, 16, 2, "fp32", 0.0)])
def test_serving_results_equal_alone_and_in_the_mix(PVFinder, weights, graphs, copy, max_batch, inflight,
                                                    precision, lead, request):
    """Zero-copy slots (mapped staging, one graph per slot with the count read on the
    device), the copy form's per-bucket graphs (a batch of k events runs the graph of the
    next bucket with the missing events empty; 24 is a bucket of its own) and stream
    launches give every request the result it has alone."""
    store = synth.generate_uneven(40, 21)
    max_pv = 96
    kw = {}
    if precision == "fp8":
        cal = synth.generate_standard(512, 1)
        pc = PVFinder(weights, precision="bf16", max_events=512, max_pv_per_event=8)
        kw["fp8_act_scales"] = pc.calibrate(*to_cuda(cal))
        pc.close()
    pv = PVFinder(weights, precision=precision, max_events=32, max_pv_per_event=max_pv, **kw)
    rng = np.random.default_rng(5)
    n = 300
    arrivals = np.cumsum(rng.exponential(1e9 / 60000.0, n)).astype(np.int64)   # 60k events/s
    req = rng.integers(0, store.n_events, n).astype(np.int32)
    done, cnt, batches, z = pv.serve_replay(store, arrivals, req, max_batch=max_batch,
                                            max_inflight=inflight, want_z=True, graphs=graphs,
                                            copy=copy, launch_lead_us=lead)
    assert batches >= n // max_batch and np.all(done >= arrivals)
    ref_cnt, ref_z = alone(pv, store, max_pv)
    np.testing.assert_array_equal(cnt, ref_cnt[req])
    for i in range(n):
        k = min(cnt[i], max_pv)
        np.testing.assert_array_equal(z[i, :k], ref_z[req[i], :k])
    lat_us = (done - arrivals) / 1000.0
    print("serving latency p50/p99 us:", np.percentile(lat_us, 50), np.percentile(lat_us, 99),
          "batches", batches)

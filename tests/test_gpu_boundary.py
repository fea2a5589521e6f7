"""Boundary tracks (§3: a track on an interval boundary belongs to two intervals) through
the C ABI, against the FP64 oracle with the same width.

Which slices an entry fills is an integer decision taken in float32 on both sides, so
the set of filled slices must match exactly; the values carry each form's usual bar.
"""

import os

import numpy as np
import pytest

import oracle
import synth
from tests.helpers import pv_agreement, to_cuda

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NTHREADS = os.cpu_count() or 1
MAX_PV = 1024
EDGE = 0.5


@pytest.fixture(scope="module")
def PVFinder():
    from paper_2602_19959_gb300 import build, PVFinder
    build()
    return PVFinder


@pytest.fixture(scope="module")
def weights():
    return synth.he_weights(0, bias_std=0.05)


@pytest.fixture(scope="module")
def ev16():
    return synth.generate_standard(16, 0)


@pytest.fixture(scope="module")
def ref16(weights, ev16):
    return oracle.infer(weights, ev16.features, ev16.offsets, max_pv=MAX_PV, want_hist=True,
                        want_logit=True, nthreads=NTHREADS, edge_mm=EDGE)


def run_full(pv, batch):
    feats, offs = to_cuda(batch)
    n = batch.n_events
    hist = torch.zeros((n, 4000), dtype=torch.float32, device="cuda")
    logit = torch.zeros((n, 4000), dtype=torch.float32, device="cuda")
    z, c = pv.infer(feats, offs, hist=hist, logit=logit)
    torch.cuda.synchronize()
    return dict(z=z.cpu().numpy(), count=c.cpu().numpy(), hist=hist.cpu().numpy(),
                logit=logit.cpu().numpy())


def rel_err(got, want):
    return max(np.max(np.abs(got[e].astype(np.float64) - want[e])) / max(np.max(np.abs(want[e])), 1e-30)
               for e in range(want.shape[0]))


def single_track_events(edge):
    """One event per track: for every slice, tracks at the two decision edges (zr = edge,
    zr = 10 - edge), one float32 ulp either side of each, and the slice's middle."""
    rng = np.random.default_rng(3)
    zs = []
    for s in range(40):
        lo = np.float32(-100 + 10 * s + edge)
        hi = np.float32(-100 + 10 * s + 10 - edge)
        for z in (lo, hi):
            zs += [z, np.nextafter(z, np.float32(-1e9)), np.nextafter(z, np.float32(1e9))]
        zs.append(np.float32(-95 + 10 * s))
    n = len(zs)
    f = np.zeros((9, n), np.float32)
    f[0] = rng.normal(0, 0.05, n)
    f[1] = rng.normal(0, 0.05, n)
    f[2] = np.asarray(zs, np.float32)
    f[3] = rng.normal(0, 0.15, n)
    f[4] = rng.normal(0, 0.15, n)
    f[5:8] = rng.lognormal(np.log(0.05), 0.5, (3, n))
    f[8] = rng.uniform(0, 1, n)
    return synth.EventBatch(features=f, offsets=np.arange(n + 1, dtype=np.int32),
                            n_pv=np.zeros(n, np.int32), pv_z=np.zeros(0))


def filled_slices(hist):
    return (hist.reshape(hist.shape[0], 40, 100) != 0).any(axis=2)


def test_fp32_end_to_end_matches_oracle(PVFinder, weights, ev16, ref16):
    pv = PVFinder(weights, precision="fp32", max_events=16, max_pv_per_event=MAX_PV, boundary_mm=EDGE)
    r = run_full(pv, ev16)
    plain = oracle.infer(weights, ev16.features, ev16.offsets, want_hist=True, nthreads=NTHREADS)
    assert np.any(ref16["hist"] != plain["hist"])             # the width changes the histogram
    np.testing.assert_array_equal(r["hist"] == 0, ref16["hist"] == 0)
    assert rel_err(r["hist"], ref16["hist"]) <= 1e-4
    assert rel_err(r["logit"], ref16["logit"]) <= 1e-4
    a = pv_agreement(ref16["pv_z"], ref16["pv_count"], r["z"], r["count"], ref16["logit"],
                     r["logit"])
    print("fp32 boundary agreement", a)
    assert a["max_dz"] <= 0.1 and a["exempt"] == 1.0 and a["strict"] >= 0.99
    assert pv.device_status() == 0


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_second_slice_decision_is_exact(PVFinder, weights, precision):
    """Both front kernels (CUDA-core and tcgen05) fill exactly the oracle's slices for
    tracks on and one ulp around every decision edge."""
    b = single_track_events(EDGE)
    pv = PVFinder(weights, precision=precision, max_events=b.n_events, max_pv_per_event=8,
                  boundary_mm=EDGE)
    feats, offs = to_cuda(b)
    hist = torch.full((b.n_events, 4000), -1.0, dtype=torch.float32, device="cuda")
    pv.stage_histogram(feats, offs, hist)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()
    ref = oracle.infer(weights, b.features, b.offsets, want_hist=True, nthreads=NTHREADS, edge_mm=EDGE)
    got, want = filled_slices(h), filled_slices(ref["hist"])
    np.testing.assert_array_equal(got, want)
    n2 = int(want.sum()) - b.n_events
    assert 40 <= n2 <= 160                                       # boundary tracks exist
    assert rel_err(h, ref["hist"]) <= (1e-4 if precision == "fp32" else 3e-2)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_every_track_a_boundary_track_at_capacity(PVFinder, weights, precision):
    """An event of max_tracks tracks, all in the boundary band: twice as many sorted
    entries as tracks, the most the plan holds."""
    rng = np.random.default_rng(12)
    n = 600
    s = rng.integers(1, 39, n)
    zr = np.where(rng.uniform(size=n) < 0.5, rng.uniform(0, EDGE * 0.9, n), rng.uniform(10 - EDGE * 0.9, 9.99, n))
    f = np.zeros((9, n), np.float32)
    f[2] = (-100 + 10 * s + zr).astype(np.float32)
    f[5:8] = 0.05
    b = synth.EventBatch(features=f, offsets=np.array([0, n], np.int32), n_pv=np.zeros(1, np.int32),
                         pv_z=np.zeros(0))
    pv = PVFinder(weights, precision=precision, max_events=1, max_tracks_per_event=n,
                  max_pv_per_event=MAX_PV, boundary_mm=EDGE)
    r = run_full(pv, b)
    ref = oracle.infer(weights, b.features, b.offsets, max_pv=MAX_PV, want_hist=True, nthreads=1,
                       edge_mm=EDGE)
    secs = sum(oracle.second_slice(z, oracle.slice_index(z)[0], EDGE) >= 0 for z in f[2])
    assert secs == n
    np.testing.assert_array_equal(r["hist"] == 0, ref["hist"] == 0)
    assert rel_err(r["hist"], ref["hist"]) <= (1e-4 if precision == "fp32" else 3e-2)
    assert r["count"][0] >= 0 and pv.device_status() == 0


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_deterministic_and_batch_invariant(PVFinder, weights, ev16, precision):
    pv = PVFinder(weights, precision=precision, max_events=16, max_pv_per_event=MAX_PV, boundary_mm=EDGE)
    r1 = run_full(pv, ev16)
    r2 = run_full(pv, ev16)
    for k in ("hist", "logit", "count"):
        np.testing.assert_array_equal(r1[k], r2[k])
    rs = run_full(pv, ev16.subset(4, 9))
    for k in ("hist", "logit", "count"):
        np.testing.assert_array_equal(rs[k], r1[k][4:9])


@pytest.mark.parametrize("precision,hist_tol,logit_tol", [("bf16", 3e-2, 5e-2), ("fp16", 4e-3, 1e-2)])
def test_tensor_core_forms_against_oracle(PVFinder, weights, ev16, ref16, precision, hist_tol, logit_tol):
    pv = PVFinder(weights, precision=precision, max_events=16, max_pv_per_event=MAX_PV, boundary_mm=EDGE)
    r = run_full(pv, ev16)
    np.testing.assert_array_equal(r["hist"] == 0, ref16["hist"] == 0)
    he, le = rel_err(r["hist"], ref16["hist"]), rel_err(r["logit"], ref16["logit"])
    a = pv_agreement(ref16["pv_z"], ref16["pv_count"], r["z"], r["count"], ref16["logit"],
                     r["logit"])
    print(f"{precision} boundary: hist err {he:.2e} logit err {le:.2e} agreement {a}")
    assert he <= hist_tol and le <= logit_tol
    assert a["max_dz"] <= 0.1 and a["exempt"] == 1.0


def test_fp8_form_against_oracle(PVFinder, weights, ev16, ref16):
    """FP8: the FC runs on bf16 operands (histogram bound as BF16), the UNet in e4m3 with
    calibrated scales (logit bound 20% of the maximum, as without boundary tracks)."""
    cal = synth.generate_standard(512, 1)
    pc = PVFinder(weights, precision="bf16", max_events=512, max_pv_per_event=8)
    feats, offs = to_cuda(cal)
    scales = pc.calibrate(feats, offs)
    pc.close()
    pv = PVFinder(weights, precision="fp8", max_events=16, max_pv_per_event=MAX_PV,
                  fp8_act_scales=scales, boundary_mm=EDGE)
    r = run_full(pv, ev16)
    np.testing.assert_array_equal(r["hist"] == 0, ref16["hist"] == 0)
    he, le = rel_err(r["hist"], ref16["hist"]), rel_err(r["logit"], ref16["logit"])
    a = pv_agreement(ref16["pv_z"], ref16["pv_count"], r["z"], r["count"], ref16["logit"],
                     r["logit"])
    print(f"fp8 boundary: hist err {he:.2e} logit err {le:.2e} agreement {a}")
    assert he <= 3e-2 and le <= 0.2
    assert a["max_dz"] <= 0.1 and a["exempt"] == 1.0
    assert pv.device_status() == 0

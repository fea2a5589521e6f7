"""GPU parity of the plain float32 form against the FP64 oracle, through the C ABI.

Bars: per-bin |err| <= 1e-4 * max(bin) for the histogram and the UNet output, and the
same PV list with each z within one bin (0.1 mm), where a PV that is present on one
side only is accepted only if the oracle's decision there is within rounding of
flipping (see tests/helpers.pv_agreement). Integer work (slices, counts, bypass
decisions) must match exactly; results must be bitwise reproducible and identical for
an event alone or inside any batch.
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


@pytest.fixture(scope="module")
def lib():
    from paper_2602_19959_gb300 import build
    build()
    from paper_2602_19959_gb300 import PVFinder
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
                        want_logit=True, nthreads=NTHREADS)


@pytest.fixture(scope="module")
def pv16(lib, weights):
    return lib(weights, precision="fp32", max_events=64, max_pv_per_event=MAX_PV)


def run_full(pv, batch):
    feats, offs = to_cuda(batch)
    n = batch.n_events
    hist = torch.zeros((n, 4000), dtype=torch.float32, device="cuda")
    logit = torch.zeros((n, 4000), dtype=torch.float32, device="cuda")
    z, c = pv.infer(feats, offs, hist=hist, logit=logit)
    torch.cuda.synchronize()
    return dict(z=z.cpu().numpy(), count=c.cpu().numpy(), hist=hist.cpu().numpy(),
                logit=logit.cpu().numpy())


def assert_per_bin(got, want, rel=1e-4):
    for e in range(want.shape[0]):
        scale = max(np.max(np.abs(want[e])), 1e-30)
        err = np.max(np.abs(got[e].astype(np.float64) - want[e]))
        assert err <= rel * scale, (e, err, scale)


def test_histogram_matches_oracle(pv16, ev16, ref16):
    feats, offs = to_cuda(ev16)
    hist = torch.zeros((16, 4000), dtype=torch.float32, device="cuda")
    pv16.stage_histogram(feats, offs, hist)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()
    assert_per_bin(h, ref16["hist"])
    # empty slices are exactly zero on both sides
    np.testing.assert_array_equal(h == 0, ref16["hist"] == 0)


def edge_batch():
    """Events exercising the integer edge cases of slicing and sorting."""
    rng = np.random.default_rng(42)
    events = []

    def ev(z, extra=None):
        n = len(z)
        f = np.zeros((9, n), np.float32)
        f[0] = rng.normal(0, 0.05, n)
        f[1] = rng.normal(0, 0.05, n)
        f[2] = np.asarray(z, np.float32)
        f[3] = rng.normal(0, 0.15, n)
        f[4] = rng.normal(0, 0.15, n)
        f[5:8] = rng.lognormal(np.log(0.05), 0.5, (3, n))
        f[8] = rng.uniform(0, 1, n)
        if extra:
            extra(f)
        events.append(f)

    ev([])                                                     # empty event
    ev([12.3])                                                 # single track
    edges = [np.float32(-100 + 10 * s) for s in range(40)]
    around = []
    for z in edges:
        around += [z, np.nextafter(z, np.float32(-1e9)), np.nextafter(z, np.float32(1e9))]
    ev(around)                                                 # exact slice edges and +-1 ulp
    ev([-100.0001, 300.0, 1e6, -1e6, 5.0, 15.0])               # out-of-range z
    def bad(f):
        f[4, 0] = np.nan
        f[6, 1] = np.inf
        f[2, 2] = np.nan
    ev([1.0, 2.0, 3.0, 4.0], bad)                              # non-finite features
    ev(rng.normal(42.0, 0.05, 300))                            # 300 tracks in one slice
    ev(rng.uniform(-100, 300, 2000))                           # many chunks, all slices
    ev(np.concatenate([rng.normal(-95, 0.1, 129), rng.normal(205, 0.1, 127)]))  # chunk edge
    feats = np.concatenate(events, axis=1)
    counts = [f.shape[1] for f in events]
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    return synth.EventBatch(features=np.ascontiguousarray(feats), offsets=offsets,
                            n_pv=np.zeros(len(events), np.int32), pv_z=np.zeros(0))


def test_histogram_edge_cases(pv16, weights):
    b = edge_batch()
    ref = oracle.infer(weights, b.features, b.offsets, max_pv=MAX_PV, want_hist=True,
                       nthreads=NTHREADS)
    feats, offs = to_cuda(b)
    hist = torch.full((b.n_events, 4000), -1.0, dtype=torch.float32, device="cuda")
    pv16.stage_histogram(feats, offs, hist)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()
    # which bins are touched is an integer decision: must match exactly
    np.testing.assert_array_equal(h != 0, ref["hist"] != 0)
    assert np.all(h[0] == 0) and np.all(h[3][:100] == 0)
    assert_per_bin(h, ref["hist"])


def test_unet_matches_oracle_on_same_histogram(pv16, weights, ref16):
    h32 = ref16["hist"].astype(np.float32)
    hist = torch.from_numpy(h32).cuda()
    logit = torch.zeros_like(hist)
    pv16.stage_unet(hist, logit)
    torch.cuda.synchronize()
    f = logit.cpu().numpy()
    want = np.stack([oracle.unet(weights, h32[e].astype(np.float64))[0] for e in range(16)])
    assert_per_bin(f, want)
    p, pw = 1 / (1 + np.exp(-f.astype(np.float64))), 1 / (1 + np.exp(-want))
    assert np.max(np.abs(p - pw)) <= 1e-4


def test_peaks_match_oracle_on_same_logits(pv16, ref16):
    f32 = ref16["logit"].astype(np.float32)
    z, c = pv16.stage_peaks(torch.from_numpy(f32).cuda())
    torch.cuda.synchronize()
    z, c = z.cpu().numpy(), c.cpu().numpy()
    for e in range(16):
        n, zr, bins = oracle.peaks(f32[e].astype(np.float64), max_pv=MAX_PV)
        assert c[e] == n                      # same float32 values: identical decisions
        np.testing.assert_allclose(z[e, :n], zr, rtol=0, atol=2e-4)


def test_peaks_edge_cases(pv16):
    f = np.full((4, 4000), -30.0, np.float32)
    f[0, [0, 3999]] = 2.0                       # both ends
    f[1, 2000:2003] = 3.0                       # plateau: leftmost wins
    f[2, [500, 505, 700, 706]] = [4.0, 3.0, 4.0, 3.0]   # 5 apart suppressed, 6 apart kept
    f[3, 10::7] = 1.0                           # 570 equal peaks 7 apart
    z, c = pv16.stage_peaks(torch.from_numpy(f).cuda())
    torch.cuda.synchronize()
    c = c.cpu().numpy()
    z = z.cpu().numpy()
    for e in range(4):
        n, zr, _ = oracle.peaks(f[e].astype(np.float64), max_pv=MAX_PV)
        assert c[e] == n
        np.testing.assert_allclose(z[e, :n], zr, atol=2e-4)
    assert c[1] == 1 and c[2] == 3 and c[3] == len(range(10, 4000, 7))


def test_end_to_end_matches_oracle(pv16, ev16, ref16):
    r = run_full(pv16, ev16)
    assert_per_bin(r["hist"], ref16["hist"])
    assert_per_bin(r["logit"], ref16["logit"])
    a = pv_agreement(ref16["pv_z"], ref16["pv_count"], r["z"], r["count"], ref16["logit"],
                     r["logit"])
    print("fp32 agreement", a)
    assert a["max_dz"] <= 0.1
    assert a["exempt"] == 1.0
    assert a["strict"] >= 0.99


def test_bitwise_reproducible_and_batch_invariant(pv16, ev16):
    r1 = run_full(pv16, ev16)
    r2 = run_full(pv16, ev16)
    for k in ("hist", "logit", "count"):
        np.testing.assert_array_equal(r1[k], r2[k])
    # event subset alone, and events in reverse order
    sub = ev16.subset(5, 9)
    rs = run_full(pv16, sub)
    for k in ("hist", "logit", "count"):
        np.testing.assert_array_equal(rs[k], r1[k][5:9])
    rev = synth.concat_batches([ev16.subset(e, e + 1) for e in range(15, -1, -1)])
    rr = run_full(pv16, rev)
    for k in ("hist", "logit", "count"):
        np.testing.assert_array_equal(rr[k][::-1], r1[k])
    for e in range(16):
        n = r1["count"][e]
        np.testing.assert_array_equal(rr["z"][15 - e, :n], r1["z"][e, :n])


def test_bypassed_events_and_device_status(lib, weights, ev16):
    pv = lib(weights, precision="fp32", max_events=16, max_pv_per_event=MAX_PV,
             max_tracks_per_event=250)
    clean = run_full(pv, ev16)
    assert pv.device_status() == 16           # events with > 250 tracks were bypassed
    big = ev16.tracks_per_event() > 250
    assert big.any() and np.all(clean["count"][big] == -1) and np.all(clean["count"][~big] >= 0)
    bad = synth.EventBatch(ev16.features, ev16.offsets.copy(), ev16.n_pv, ev16.pv_z)
    bad.offsets[4] = bad.offsets[3] - 5       # event 3 decreasing
    r = run_full(pv, bad)
    assert r["count"][3] == -1
    keep = [e for e in range(16) if e not in (3, 4) and not big[e]]
    np.testing.assert_array_equal(r["logit"][keep], clean["logit"][keep])
    assert pv.device_status() == 16
    assert pv.device_status() == 0            # reading clears


def test_truncation_and_chunking(lib, weights, ev16, ref16):
    pv = lib(weights, precision="fp32", max_events=16, max_pv_per_event=8, chunk_events=3)
    r = run_full(pv, ev16)
    assert pv.device_status() == 17
    full = run_full(lib(weights, precision="fp32", max_events=16, max_pv_per_event=MAX_PV), ev16)
    np.testing.assert_array_equal(r["count"], full["count"])
    np.testing.assert_array_equal(r["logit"], full["logit"])
    for e in range(16):
        np.testing.assert_array_equal(r["z"][e], full["z"][e, :8])


def test_zero_events(pv16, ev16):
    feats, offs = to_cuda(ev16)
    z, c = pv16.alloc_outputs(1)
    pv16.infer(feats, offs[:1], n_events=0, out=(z, c))
    torch.cuda.synchronize()


def test_full_size_sampled(lib, weights):
    """The 1000-event workload in the bench's configuration; oracle on sampled events."""
    b = synth.generate_standard(1000, 1)
    # 672 slots: the rule keeps peaks >= 6 bins apart, so no event can have more than 667
    pv = lib(weights, precision="fp32", max_events=1000, max_pv_per_event=672)
    r = run_full(pv, b)
    assert np.all(r["count"] >= 0)
    sample = [0, 1, 499, 500, 998, 999]
    sb = synth.concat_batches([b.subset(e, e + 1) for e in sample])
    ref = oracle.infer(weights, sb.features, sb.offsets, max_pv=672, want_hist=True,
                       want_logit=True, nthreads=NTHREADS)
    assert_per_bin(r["hist"][sample], ref["hist"])
    assert_per_bin(r["logit"][sample], ref["logit"])
    a = pv_agreement(ref["pv_z"], ref["pv_count"], r["z"][sample], r["count"][sample], ref["logit"],
                     r["logit"][sample])
    assert a["exempt"] == 1.0
    assert pv.device_status() == 0
    for e in range(1000):
        n = r["count"][e]
        zz = r["z"][e, :n]
        assert np.all(np.diff(zz) > 0) and np.all(zz >= -100) and np.all(zz < 300)


# ---------------------------------------------------------------- wide UNet (base width 32)
# §5's channel-count axis: every UNet level twice as wide (32/64/128/256), four times the
# MACs. Built in the float32 form; the same bars as the width-16 network.

@pytest.fixture(scope="module")
def wide_weights():
    return synth.he_weights(0, bias_std=0.05, c0=32)


@pytest.fixture(scope="module")
def wide_ref(wide_weights):
    ev = synth.generate_standard(8, 0)
    return ev, oracle.infer(wide_weights, ev.features, ev.offsets, max_pv=MAX_PV, want_hist=True,
                            want_logit=True, nthreads=NTHREADS)


@pytest.fixture(scope="module")
def wide_pv(lib, wide_weights):
    return lib(wide_weights, precision="fp32", max_events=8, max_pv_per_event=MAX_PV)


def test_wide_unet_stage_matches_oracle(wide_pv, wide_weights, wide_ref):
    _, ref = wide_ref
    h32 = ref["hist"].astype(np.float32)
    logit = torch.zeros((8, 4000), dtype=torch.float32, device="cuda")
    wide_pv.stage_unet(torch.from_numpy(h32).cuda(), logit)
    torch.cuda.synchronize()
    want = np.stack([oracle.unet(wide_weights, h32[e].astype(np.float64))[0] for e in range(8)])
    assert_per_bin(logit.cpu().numpy(), want)


def test_wide_end_to_end_matches_oracle(wide_pv, wide_ref):
    ev, ref = wide_ref
    r = run_full(wide_pv, ev)
    np.testing.assert_array_equal(r["hist"] == 0, ref["hist"] == 0)
    assert_per_bin(r["hist"], ref["hist"])
    assert_per_bin(r["logit"], ref["logit"])
    a = pv_agreement(ref["pv_z"], ref["pv_count"], r["z"], r["count"], ref["logit"],
                     r["logit"])
    print("wide fp32 agreement", a)
    assert a["max_dz"] <= 0.1 and a["exempt"] == 1.0 and a["strict"] >= 0.99
    assert wide_pv.device_status() == 0


def test_wide_bitwise_reproducible_batch_invariant_and_chunked(lib, wide_pv, wide_weights, wide_ref):
    ev, _ = wide_ref
    r1 = run_full(wide_pv, ev)
    r2 = run_full(wide_pv, ev)
    rs = run_full(wide_pv, ev.subset(2, 5))
    chunked = lib(wide_weights, precision="fp32", max_events=8, chunk_events=3, max_pv_per_event=MAX_PV)
    rc = run_full(chunked, ev)
    for k in ("hist", "logit", "count"):
        np.testing.assert_array_equal(r1[k], r2[k])
        np.testing.assert_array_equal(rs[k], r1[k][2:5])
        np.testing.assert_array_equal(rc[k], r1[k])



# ---------------------------------------------------------------- per-interval layout (§3)
# Each of the 40 intervals runs the UNet as its own 104-bin sequence (two zero bins on each
# side); its 100 central logits fill the interval's bins. Built in the float32 form.

@pytest.fixture(scope="module")
def iv_ref(weights, ev16):
    return oracle.infer(weights, ev16.features, ev16.offsets, max_pv=MAX_PV, want_hist=True,
                        want_logit=True, nthreads=NTHREADS, per_interval=True)


@pytest.fixture(scope="module")
def iv_pv(lib, weights):
    return lib(weights, precision="fp32", max_events=16, max_pv_per_event=MAX_PV, per_interval=True)


def test_per_interval_unet_stage_matches_oracle(iv_pv, weights, ref16):
    h32 = ref16["hist"].astype(np.float32)
    logit = torch.zeros((16, 4000), dtype=torch.float32, device="cuda")
    iv_pv.stage_unet(torch.from_numpy(h32).cuda(), logit)
    torch.cuda.synchronize()
    want = np.stack([oracle.unet_intervals(weights, h32[e].astype(np.float64))[0] for e in range(16)])
    assert_per_bin(logit.cpu().numpy(), want)


def test_per_interval_end_to_end_matches_oracle(iv_pv, ev16, iv_ref, ref16):
    r = run_full(iv_pv, ev16)
    assert_per_bin(r["hist"], ref16["hist"])            # the histogram does not depend on the layout
    assert_per_bin(r["logit"], iv_ref["logit"])
    assert np.max(np.abs(iv_ref["logit"] - ref16["logit"])) > 1e-3      # a different network output
    a = pv_agreement(iv_ref["pv_z"], iv_ref["pv_count"], r["z"], r["count"], iv_ref["logit"],
                     r["logit"])
    print("per-interval fp32 agreement", a)
    assert a["max_dz"] <= 0.1 and a["exempt"] == 1.0 and a["strict"] >= 0.99
    assert iv_pv.device_status() == 0


def test_per_interval_bitwise_batch_invariant_and_chunked(lib, iv_pv, weights, ev16):
    r1 = run_full(iv_pv, ev16)
    r2 = run_full(iv_pv, ev16)
    rs = run_full(iv_pv, ev16.subset(6, 10))
    chunked = lib(weights, precision="fp32", max_events=16, chunk_events=5, max_pv_per_event=MAX_PV,
                  per_interval=True)
    rc = run_full(chunked, ev16)
    for k in ("hist", "logit", "count"):
        np.testing.assert_array_equal(r1[k], r2[k])
        np.testing.assert_array_equal(rs[k], r1[k][6:10])
        np.testing.assert_array_equal(rc[k], r1[k])


def test_per_interval_with_boundary_tracks_matches_oracle(lib, weights, ev16):
    """§3's combination: intervals processed on their own, boundary tracks in two."""
    ref = oracle.infer(weights, ev16.features, ev16.offsets, max_pv=MAX_PV, want_hist=True,
                       want_logit=True, nthreads=NTHREADS, per_interval=True, edge_mm=0.5)
    pv = lib(weights, precision="fp32", max_events=16, max_pv_per_event=MAX_PV, per_interval=True,
             boundary_mm=0.5)
    r = run_full(pv, ev16)
    assert_per_bin(r["hist"], ref["hist"])
    assert_per_bin(r["logit"], ref["logit"])
    a = pv_agreement(ref["pv_z"], ref["pv_count"], r["z"], r["count"], ref["logit"],
                     r["logit"])
    assert a["max_dz"] <= 0.1 and a["exempt"] == 1.0 and a["strict"] >= 0.99



def test_end_to_end_closed_form(lib):
    """All four steps against hand-derived values (the oracle pin of the same name): zero
    FC weights and the identity UNet, so each populated slice s gives one vertex at
    z = -100 + (100 s + 50.5) * 0.1."""
    from tests.test_oracle_pins import identity_unet_weights
    a, c = 0.5, -6.0
    w = identity_unet_weights(a, c)
    j = np.arange(100)
    b6 = (3.0 - (j - 50.0) ** 2 / 20.0).astype(np.float32)
    w["fc6"] = (w["fc6"][0], b6)
    counts = {3: 1, 7: 2, 20: 5, 39: 3}
    z = [np.float32(-100 + 10 * s + 4.2) for s, n in counts.items() for _ in range(n)]
    f = np.random.default_rng(30).normal(0, 1, (9, len(z))).astype(np.float32)
    f[2] = z
    b = synth.EventBatch(features=f, offsets=np.array([0, len(z)], np.int32),
                         n_pv=np.zeros(1, np.int32), pv_z=np.zeros(0))
    pv = lib(w, precision="fp32", max_events=1, max_pv_per_event=64)
    r = run_full(pv, b)
    sp = np.logaddexp(0.0, b6.astype(np.float64))
    want_hist = np.zeros(4000)
    for s, n in counts.items():
        want_hist[100 * s:100 * s + 100] = n * sp
    assert_per_bin(r["hist"], want_hist[None])
    assert_per_bin(r["logit"], (a * want_hist + c)[None])
    assert r["count"][0] == len(counts)
    want_z = [-100.0 + (100 * s + 50 + 0.5) * 0.1 for s in sorted(counts)]
    np.testing.assert_allclose(r["z"][0, :len(counts)], want_z, rtol=0, atol=1e-3)
    assert pv.device_status() == 0

"""GPU checks of the tensor-core (tcgen05) forms through the C ABI.

1. Kernel wiring: the BF16 UNet against a float64 emulation that rounds to bf16 at
   exactly the points where the kernels store bf16 (tests/ref_torch64.unet_quantized):
   only float32-accumulation differences and the occasional one-ulp rounding flip remain.
2. Against the FP64 oracle: per-bin error of the logits (reported and bounded) and the
   PV-list agreement, strict and with the near-tie exemption computed from the measured
   per-bin logit differences (paper_2602_19959_gb300.agreement).
3. Determinism and batch invariance, as for the FP32 form.
"""

import os

import numpy as np
import pytest

import oracle
import synth
from tests import ref_torch64 as ref
from tests.helpers import pv_agreement, to_cuda

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
NTHREADS = os.cpu_count() or 1
MAX_PV = 672


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
                        want_logit=True, nthreads=NTHREADS)


@pytest.fixture(scope="module")
def bf16(PVFinder, weights):
    return PVFinder(weights, precision="bf16", max_events=64, max_pv_per_event=MAX_PV)


def run_full(pv, batch):
    feats, offs = to_cuda(batch)
    n = batch.n_events
    hist = torch.zeros((n, 4000), dtype=torch.float32, device="cuda")
    logit = torch.zeros((n, 4000), dtype=torch.float32, device="cuda")
    z, c = pv.infer(feats, offs, hist=hist, logit=logit)
    torch.cuda.synchronize()
    r = dict(z=z.cpu().numpy(), count=c.cpu().numpy(), hist=hist.cpu().numpy(),
             logit=logit.cpu().numpy())
    assert np.all(np.isfinite(r["hist"])) and np.all(np.isfinite(r["logit"]))
    return r


def test_bf16_unet_wiring_matches_quantised_emulation(bf16, weights, ref16):
    h32 = ref16["hist"].astype(np.float32)
    logit = torch.zeros((16, 4000), dtype=torch.float32, device="cuda")
    bf16.stage_unet(torch.from_numpy(h32).cuda(), logit)
    torch.cuda.synchronize()
    f = logit.cpu().numpy().astype(np.float64)
    for e in range(4):
        want = ref.unet_quantized(weights, h32[e].astype(np.float64), ref.q_bf16)
        scale = np.max(np.abs(want))
        d = np.abs(f[e] - want) / scale
        print(f"event {e}: median {np.median(d):.2e} p99 {np.quantile(d, 0.99):.2e} max {d.max():.2e}")
        assert np.median(d) <= 1e-4
        assert np.quantile(d, 0.99) <= 2e-3
        assert d.max() <= 2e-2


def test_bf16_fc_wiring_matches_quantised_emulation(bf16, weights, ev16):
    r = run_full(bf16, ev16)
    for e in range(6):
        feats = ev16.features[:, ev16.offsets[e]:ev16.offsets[e + 1]]
        want = ref.histogram_quantized(weights, feats, ref.q_bf16)
        scale = np.max(np.abs(want))
        d = np.abs(r["hist"][e] - want) / scale
        print(f"fc event {e}: median {np.median(d):.2e} max {d.max():.2e}")
        assert np.median(d) <= 1e-5
        assert d.max() <= 2e-3
        np.testing.assert_array_equal(r["hist"][e] == 0, want == 0)


def test_bf16_histogram_against_oracle(bf16, ev16, ref16):
    """bf16 FC (8-bit mantissas, six layers): per-bin error within 3% of the event max."""
    r = run_full(bf16, ev16)
    worst = 0.0
    for e in range(16):
        scale = np.max(np.abs(ref16["hist"][e]))
        err = np.max(np.abs(r["hist"][e] - ref16["hist"][e])) / scale
        worst = max(worst, err)
        assert err <= 3e-2
    print("bf16 histogram per-bin err / max:", worst)


def test_bf16_against_oracle(bf16, ev16, ref16):
    r = run_full(bf16, ev16)
    rel = [np.max(np.abs(r["logit"][e] - ref16["logit"][e])) / np.max(np.abs(ref16["logit"][e]))
           for e in range(16)]
    prob_err = np.max(np.abs(1 / (1 + np.exp(-r["logit"].astype(np.float64))) -
                             1 / (1 + np.exp(-ref16["logit"]))))
    a = pv_agreement(ref16["pv_z"], ref16["pv_count"], r["z"], r["count"], ref16["logit"],
                     r["logit"])
    print("bf16 per-bin logit err / max:", max(rel), "prob err:", prob_err, "agreement:", a)
    assert max(rel) <= 0.05
    assert a["max_dz"] <= 0.1
    # every disagreement is a decision the measured per-bin differences can flip; BF16 misses
    # the 99.9% strict bar (measured 99.15% on these events), the guard below catches a drop
    assert a["exempt"] == 1.0
    assert a["strict"] >= 0.985


def test_bf16_deterministic_and_batch_invariant(bf16, ev16):
    r1 = run_full(bf16, ev16)
    r2 = run_full(bf16, ev16)
    for k in ("hist", "logit", "count"):
        np.testing.assert_array_equal(r1[k], r2[k])
    rs = run_full(bf16, ev16.subset(3, 7))
    for k in ("hist", "logit", "count"):
        np.testing.assert_array_equal(rs[k], r1[k][3:7])
    rev = synth.concat_batches([ev16.subset(e, e + 1) for e in range(15, -1, -1)])
    rr = run_full(bf16, rev)
    np.testing.assert_array_equal(rr["logit"][::-1], r1["logit"])


def test_bf16_full_size_sampled(PVFinder, weights):
    b = synth.generate_standard(1000, 1)
    pv = PVFinder(weights, precision="bf16", max_events=1000, max_pv_per_event=MAX_PV)
    r = run_full(pv, b)
    assert pv.device_status() == 0
    sample = [0, 999]
    sb = synth.concat_batches([b.subset(e, e + 1) for e in sample])
    rr = oracle.infer(weights, sb.features, sb.offsets, max_pv=MAX_PV, want_logit=True,
                      nthreads=NTHREADS)
    for i, e in enumerate(sample):
        assert np.max(np.abs(r["logit"][e] - rr["logit"][i])) <= 0.05 * np.max(np.abs(rr["logit"][i]))
    assert np.all(r["count"] >= 0)


@pytest.mark.parametrize("precision", ["bf16", "fp16", "fp8"])
def test_chunked_and_repeated_launches_equal_one_launch(PVFinder, weights, precision, request):
    """One call split into UNet chunks of 16 events, and the same handle reused for
    different batch sizes, give bit for bit the results of a single launch: every kernel
    (including the encoders' tile counters, which each launch leaves at zero) starts
    from a clean state."""
    kw = {}
    if precision == "fp8":
        kw["fp8_act_scales"] = request.getfixturevalue("fp8_scales")
    b = synth.generate_uneven(48, 31)
    one = PVFinder(weights, precision=precision, max_events=48, max_pv_per_event=MAX_PV, **kw)
    chunked = PVFinder(weights, precision=precision, max_events=48, chunk_events=16,
                       max_pv_per_event=MAX_PV, **kw)
    r1 = run_full(one, b)
    rc = run_full(chunked, b)
    for k in ("hist", "logit", "count"):
        np.testing.assert_array_equal(rc[k], r1[k])
    for n in (1, 7, 48, 3):          # sizes that leave different tile counts per launch
        rs = run_full(one, b.subset(0, n))
        for k in ("hist", "logit", "count"):
            np.testing.assert_array_equal(rs[k], r1[k][:n])
    assert one.device_status() == 0 and chunked.device_status() == 0


# ---------------------------------------------------------------- FP8 (E4M3)

@pytest.fixture(scope="module")
def fp8_scales(PVFinder, weights):
    """Per-tensor activation scales from the calibration pass: 512 seeded events, disjoint
    from the test events, through a BF16 handle."""
    cal = synth.generate_standard(512, 1)
    pv = PVFinder(weights, precision="bf16", max_events=512, max_pv_per_event=8)
    feats, offs = to_cuda(cal)
    scales = pv.calibrate(feats, offs)
    pv.close()
    return scales


@pytest.fixture(scope="module")
def fp8(PVFinder, weights, fp8_scales):
    return PVFinder(weights, precision="fp8", max_events=64, max_pv_per_event=MAX_PV,
                    fp8_act_scales=fp8_scales)


def test_fp8_calibration_scales(fp8_scales):
    assert np.all(np.isfinite(fp8_scales)) and np.all(fp8_scales > 0)
    assert np.all(fp8_scales[7:] == 1.0)
    assert np.all(fp8_scales[:7] != 1.0)
    print("fp8 act scales:", fp8_scales[:7])


def _poison_shared_memory():
    """Leaves NaN bit patterns in shared memory of every SM (a float32 fill of NaNs sized
    to run on all SMs), so that a kernel reading a shared-memory row it never wrote
    produces NaN instead of a plausible number."""
    x = torch.full((152 * 64 * 1024,), float("nan"), device="cuda")
    torch.cumsum(x.view(152 * 64, 1024), dim=1)
    torch.cuda.synchronize()


def test_fp8_unet_wiring_matches_quantised_emulation(fp8, weights, ref16, fp8_scales):
    h32 = ref16["hist"].astype(np.float32)
    logit = torch.zeros((16, 4000), dtype=torch.float32, device="cuda")
    _poison_shared_memory()
    fp8.stage_unet(torch.from_numpy(h32).cuda(), logit)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(logit.cpu().numpy()))
    f = logit.cpu().numpy().astype(np.float64)
    for e in range(4):
        want = ref.unet_quantized_fp8(weights, h32[e].astype(np.float64), fp8_scales)
        scale = np.max(np.abs(want))
        d = np.abs(f[e] - want) / scale
        print(f"fp8 event {e}: median {np.median(d):.2e} p99 {np.quantile(d, 0.99):.2e} max {d.max():.2e}")
        assert np.median(d) <= 1e-3
        assert np.quantile(d, 0.99) <= 3e-2


def test_fp8_against_oracle(fp8, ev16, ref16):
    r = run_full(fp8, ev16)
    rel = [np.max(np.abs(r["logit"][e] - ref16["logit"][e])) / np.max(np.abs(ref16["logit"][e]))
           for e in range(16)]
    a = pv_agreement(ref16["pv_z"], ref16["pv_count"], r["z"], r["count"], ref16["logit"],
                     r["logit"])
    print("fp8 per-bin logit err / max:", max(rel), "agreement:", a)
    assert max(rel) <= 0.2
    assert a["max_dz"] <= 0.1
    # FP8 misses the 99.9% strict bar (measured 93.7%); every disagreement is explained by
    # the measured per-bin differences
    assert a["exempt"] == 1.0
    assert a["strict"] >= 0.9


def test_fp8_deterministic_and_batch_invariant(fp8, ev16):
    r1 = run_full(fp8, ev16)
    r2 = run_full(fp8, ev16)
    for k in ("hist", "logit", "count"):
        np.testing.assert_array_equal(r1[k], r2[k])
    rs = run_full(fp8, ev16.subset(9, 12))
    np.testing.assert_array_equal(rs["logit"], r1["logit"][9:12])


# ---------------------------------------------------------------- FP16 (the §5 proposal)
# Same kernels as BF16 with f16 operands (10 stored mantissa bits instead of 7): every
# rounding error is about 8x smaller, and the bounds below are set accordingly (the BF16
# form measures a histogram error of ~4e-3 and a logit error of ~1.3e-2 of the maximum).

@pytest.fixture(scope="module")
def fp16(PVFinder, weights):
    return PVFinder(weights, precision="fp16", max_events=64, max_pv_per_event=MAX_PV)


def test_fp16_unet_wiring_matches_quantised_emulation(fp16, weights, ref16):
    h32 = ref16["hist"].astype(np.float32)
    logit = torch.zeros((16, 4000), dtype=torch.float32, device="cuda")
    _poison_shared_memory()
    fp16.stage_unet(torch.from_numpy(h32).cuda(), logit)
    torch.cuda.synchronize()
    f = logit.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(f))
    for e in range(4):
        want = ref.unet_quantized(weights, h32[e].astype(np.float64), ref.q_fp16)
        scale = np.max(np.abs(want))
        d = np.abs(f[e] - want) / scale
        print(f"fp16 event {e}: median {np.median(d):.2e} p99 {np.quantile(d, 0.99):.2e} max {d.max():.2e}")
        assert np.median(d) <= 1e-4
        assert np.quantile(d, 0.99) <= 5e-4
        assert d.max() <= 5e-3


def test_fp16_fc_wiring_matches_quantised_emulation(fp16, weights, ev16):
    r = run_full(fp16, ev16)
    for e in range(6):
        feats = ev16.features[:, ev16.offsets[e]:ev16.offsets[e + 1]]
        want = ref.histogram_quantized(weights, feats, ref.q_fp16)
        scale = np.max(np.abs(want))
        d = np.abs(r["hist"][e] - want) / scale
        print(f"fp16 fc event {e}: median {np.median(d):.2e} max {d.max():.2e}")
        assert np.median(d) <= 1e-5
        assert d.max() <= 5e-4
        np.testing.assert_array_equal(r["hist"][e] == 0, want == 0)


def test_fp16_against_oracle(fp16, ev16, ref16):
    r = run_full(fp16, ev16)
    hist = max(np.max(np.abs(r["hist"][e] - ref16["hist"][e])) / np.max(np.abs(ref16["hist"][e]))
               for e in range(16))
    rel = max(np.max(np.abs(r["logit"][e] - ref16["logit"][e])) / np.max(np.abs(ref16["logit"][e]))
              for e in range(16))
    a = pv_agreement(ref16["pv_z"], ref16["pv_count"], r["z"], r["count"], ref16["logit"],
                     r["logit"])
    print("fp16 histogram err / max:", hist, "per-bin logit err / max:", rel, "agreement:", a)
    assert hist <= 4e-3
    assert rel <= 1e-2
    assert a["max_dz"] <= 0.1
    # the headline form: strict agreement at the 99.9% bar, and every disagreement a decision
    # the measured per-bin differences can flip
    assert a["strict"] >= 0.999
    assert a["exempt"] == 1.0


def test_fp16_deterministic_and_batch_invariant(fp16, ev16):
    r1 = run_full(fp16, ev16)
    r2 = run_full(fp16, ev16)
    for k in ("hist", "logit", "count"):
        np.testing.assert_array_equal(r1[k], r2[k])
    rs = run_full(fp16, ev16.subset(5, 11))
    for k in ("hist", "logit", "count"):
        np.testing.assert_array_equal(rs[k], r1[k][5:11])
    assert fp16.device_status() == 0


def test_fp16_full_size_sampled(PVFinder, weights):
    """The 1000-event workload in the launch configuration the bench times, checked against
    the oracle on a sample of events."""
    b = synth.generate_standard(1000, 1)
    pv = PVFinder(weights, precision="fp16", max_events=1000, max_pv_per_event=MAX_PV)
    r = run_full(pv, b)
    assert pv.device_status() == 0
    sample = [0, 500, 999]
    sb = synth.concat_batches([b.subset(e, e + 1) for e in sample])
    rr = oracle.infer(weights, sb.features, sb.offsets, max_pv=MAX_PV, want_logit=True,
                      nthreads=NTHREADS)
    for i, e in enumerate(sample):
        assert np.max(np.abs(r["logit"][e] - rr["logit"][i])) <= 1e-2 * np.max(np.abs(rr["logit"][i]))
    assert np.all(r["count"] >= 0)

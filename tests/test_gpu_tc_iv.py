"""The per-interval layout (§3: the CNN batched over the 40 intervals of an event, each run
as its own 104-bin sequence) in the tensor-core forms, through the C ABI.

1. Kernel wiring: each interval's logits against the float64 emulation with 16-bit
   rounding at every stored tensor, applied to that interval's 104-bin window.
2. Against the FP64 oracle in the same layout: per-bin logit error within the form's
   bound and PV-list agreement (strict reported; every disagreement explained by the
   measured per-bin logit differences).
3. Determinism and batch invariance.
"""

import os

import numpy as np
import pytest

import oracle
import synth
from tests import ref_torch64 as ref
from tests.helpers import logit_errors, pv_agreement, to_cuda

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
def iv_ref(weights, ev16):
    return oracle.infer(weights, ev16.features, ev16.offsets, max_pv=MAX_PV, want_hist=True,
                        want_logit=True, nthreads=NTHREADS, per_interval=True)


@pytest.fixture(scope="module")
def fp8_scales(PVFinder, weights):
    cal = synth.generate_standard(512, 1)
    pv = PVFinder(weights, precision="bf16", max_events=512, max_pv_per_event=8)
    scales = pv.calibrate(*to_cuda(cal))
    pv.close()
    return scales


def make(PVFinder, weights, precision, fp8_scales=None, n=16):
    kw = {"fp8_act_scales": fp8_scales} if precision == "fp8" else {}
    return PVFinder(weights, precision=precision, max_events=n, max_pv_per_event=MAX_PV, per_interval=True,
                    **kw)


def run_full(pv, batch):
    feats, offs = to_cuda(batch)
    n = batch.n_events
    hist = torch.zeros((n, 4000), device="cuda")
    logit = torch.zeros((n, 4000), device="cuda")
    z, c = pv.infer(feats, offs, hist=hist, logit=logit)
    torch.cuda.synchronize()
    r = dict(z=z.cpu().numpy(), count=c.cpu().numpy(), hist=hist.cpu().numpy(), logit=logit.cpu().numpy())
    assert np.all(np.isfinite(r["logit"]))
    return r


def window_logits(weights, hist, q):
    """The emulated logits of one event in the per-interval layout: each interval's 100 bins
    with two zero bins on each side, its 100 central logits."""
    out = np.zeros(4000)
    for s in range(40):
        win = np.concatenate([[0.0, 0.0], hist[100 * s:100 * s + 100], [0.0, 0.0]])
        out[100 * s:100 * s + 100] = ref.unet_quantized(weights, win, q)[2:102]
    return out


@pytest.mark.parametrize("precision,q", [("fp16", ref.q_fp16), ("bf16", ref.q_bf16)])
def test_per_interval_wiring_matches_quantised_emulation(PVFinder, weights, iv_ref, precision, q):
    pv = make(PVFinder, weights, precision)
    h32 = iv_ref["hist"].astype(np.float32)
    logit = torch.zeros((16, 4000), device="cuda")
    pv.stage_unet(torch.from_numpy(h32).cuda(), logit)
    torch.cuda.synchronize()
    f = logit.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(f))
    for e in range(3):
        want = window_logits(weights, h32[e].astype(np.float64), q)
        d = np.abs(f[e] - want) / np.max(np.abs(want))
        print(f"{precision} iv event {e}: median {np.median(d):.2e} p99 {np.quantile(d, 0.99):.2e} "
              f"max {d.max():.2e}")
        assert np.median(d) <= 1e-4
        assert d.max() <= (5e-3 if precision == "fp16" else 2e-2)


# strict agreement: FP16 at the 99.9% bar (measured 99.97%); BF16 and FP8 below it in this
# layout (measured 93.4% and 85.2% on these events), guarded against a further drop; every
# disagreement of every form must be explained by the measured per-bin differences
@pytest.mark.parametrize("precision,logit_tol,strict_min", [("fp16", 1e-2, 0.999), ("bf16", 5e-2, 0.9),
                                                            ("fp8", 0.35, 0.8)])
def test_per_interval_against_oracle(PVFinder, weights, ev16, iv_ref, fp8_scales, precision, logit_tol,
                                     strict_min):
    pv = make(PVFinder, weights, precision, fp8_scales)
    r = run_full(pv, ev16)
    assert pv.device_status() == 0
    le = logit_errors(iv_ref["logit"], r["logit"])
    a = pv_agreement(iv_ref["pv_z"], iv_ref["pv_count"], r["z"], r["count"], iv_ref["logit"], r["logit"])
    print(f"{precision} per-interval: logit err / max {le.max():.3e} agreement {a}")
    assert le.max() <= logit_tol
    assert a["max_dz"] <= 0.1 and a["exempt"] == 1.0 and a["strict"] >= strict_min


@pytest.mark.parametrize("precision", ["fp16", "fp8"])
def test_per_interval_deterministic_and_batch_invariant(PVFinder, weights, ev16, fp8_scales, precision):
    pv = make(PVFinder, weights, precision, fp8_scales)
    r1 = run_full(pv, ev16)
    r2 = run_full(pv, ev16)
    for k in ("hist", "logit", "count"):
        np.testing.assert_array_equal(r1[k], r2[k])
    rs = run_full(pv, ev16.subset(5, 9))
    for k in ("hist", "logit", "count"):
        np.testing.assert_array_equal(rs[k], r1[k][5:9])


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_per_interval_chunked_dirty_pool_and_front_shapes(PVFinder, weights, precision):
    """Every zero row of the layout (between sequences, at both event ends, in e1, p1, the
    pooled and the upsampled tensors) is written each time: 48 uneven events in chunks of
    7 (a partial last chunk), on a pool first filled by another batch, under both front
    shapes, give bit for bit the results of one unchunked launch on a fresh pool."""
    b = synth.generate_uneven(48, 13)
    other = synth.generate_uneven(48, 21)
    pv = PVFinder(weights, precision=precision, max_events=48, max_pv_per_event=MAX_PV, per_interval=True)
    want = run_full(pv, b)
    pv.close()
    for sched in ({"front": 2}, {"front": 4}):
        pc = PVFinder(weights, precision=precision, max_events=48, chunk_events=7, max_pv_per_event=MAX_PV,
                      per_interval=True, schedule=sched)
        run_full(pc, other)                      # leaves other events' activations in every slot
        got = run_full(pc, b)
        pc.close()
        for k in ("hist", "logit", "count"):
            np.testing.assert_array_equal(got[k], want[k])
        for e in range(48):
            k = min(int(want["count"][e]), MAX_PV)
            np.testing.assert_array_equal(got["z"][e, :k], want["z"][e, :k])

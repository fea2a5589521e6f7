"""The precision study on 20000 events: every form of the path against the FP64 oracle.

Workload: the standard generator, 20000 events (seed 3000), He-initialised weights with
zero biases (the benchmark's network); the FP8 activation scales come from a calibration
pass over 512 seeded events (seed 1, disjoint from these) through a BF16 handle.

Reported per form: the per-bin error of the histogram and of the logits relative to each
event's maximum (max and median over events), and the PV-list agreement, strict and with
the exemption for disagreements that the measured per-bin logit differences can explain.
Bars: FP32 within 1e-4 of the maximum per bin; FP16, the headline reduced form, at strict
agreement >= 99.9%; BF16 and FP8 are reported with their strict agreement (both below
99.9% with these random weights) and must have every disagreement explained.
"""

import json
import os

import numpy as np
import pytest

import oracle
import synth
from tests.helpers import logit_errors, pv_agreement, to_cuda

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_EVENTS = 20000
SEED = 3000
MAX_PV = 672
CHUNK = 2000
NTHREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def weights():
    return synth.he_weights(0)


@pytest.fixture(scope="module")
def events():
    return synth.generate_standard(N_EVENTS, SEED)


@pytest.fixture(scope="module")
def ref(weights, events):
    return oracle.infer(weights, events.features, events.offsets, max_pv=MAX_PV, want_hist=True,
                        want_logit=True, nthreads=NTHREADS)


@pytest.fixture(scope="module")
def PVFinder():
    from paper_2602_19959_gb300 import build, PVFinder
    build()
    return PVFinder


def run_form(PVFinder, weights, events, precision):
    kw = {}
    if precision == "fp8":
        cal = synth.generate_standard(512, 1)
        pc = PVFinder(weights, precision="bf16", max_events=512, max_pv_per_event=8)
        kw["fp8_act_scales"] = pc.calibrate(*to_cuda(cal))
        pc.close()
    pv = PVFinder(weights, precision=precision, max_events=N_EVENTS, chunk_events=CHUNK,
                  max_pv_per_event=MAX_PV, **kw)
    feats, offs = to_cuda(events)
    hist = torch.zeros((N_EVENTS, 4000), dtype=torch.float32, device="cuda")
    logit = torch.zeros((N_EVENTS, 4000), dtype=torch.float32, device="cuda")
    z, c = pv.infer(feats, offs, hist=hist, logit=logit)
    torch.cuda.synchronize()
    assert pv.device_status() == 0
    r = dict(z=z.cpu().numpy(), count=c.cpu().numpy(), hist=hist.cpu().numpy(),
             logit=logit.cpu().numpy())
    pv.close()
    del hist, logit, z, c
    torch.cuda.empty_cache()
    return r


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16", "fp8"])
def test_precision_study_20000_events(PVFinder, weights, events, ref, precision):
    r = run_form(PVFinder, weights, events, precision)
    assert np.all(np.isfinite(r["hist"])) and np.all(np.isfinite(r["logit"]))
    he = logit_errors(ref["hist"], r["hist"])
    le = logit_errors(ref["logit"], r["logit"])
    a = pv_agreement(ref["pv_z"], ref["pv_count"], r["z"], r["count"], ref["logit"], r["logit"])
    summary = {"form": precision, "events": N_EVENTS, "hist_err_max": float(he.max()),
               "hist_err_median": float(np.median(he)), "logit_err_max": float(le.max()),
               "logit_err_median": float(np.median(le)), **a}
    print("PRECISION_STUDY " + json.dumps(summary))
    assert a["max_dz"] <= 0.1
    assert a["exempt"] == 1.0
    if precision == "fp32":
        assert he.max() <= 1e-4 and le.max() <= 1e-4
        assert a["strict"] >= 0.9999
    elif precision == "fp16":
        assert he.max() <= 4e-3 and le.max() <= 1e-2
        assert a["strict"] >= 0.999
    elif precision == "bf16":
        assert he.max() <= 3e-2 and le.max() <= 5e-2
        assert a["strict"] >= 0.985
    else:
        # 3-bit mantissas: 2^-4 relative per stored tensor and about ten stored tensors in
        # the chain; measured max 0.27 and median 0.11 of the event maximum
        assert le.max() <= 0.35 and np.median(le) <= 0.15
        assert a["strict"] >= 0.85

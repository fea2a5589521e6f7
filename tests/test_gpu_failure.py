"""Failure detection on the GPU without a fault: every device-side wait of the
tensor-core kernels is bounded, and a wait that runs out makes the kernel record
PVF_ERR_TIMEOUT, drain its own copies, free its tensor memory and return. The test makes
one wait run out on purpose (a barrier that nothing arrives on, given up after 2 ms) and
checks that the status is reported and that the handle then gives exactly its earlier
results."""

import time

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


def run(pv, batch):
    feats, offs = to_cuda(batch)
    logit = torch.zeros((batch.n_events, 4000), device="cuda")
    z, c = pv.infer(feats, offs, logit=logit)
    torch.cuda.synchronize()
    return logit.cpu().numpy(), c.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp16", "bf16", "fp8"])
def test_bounded_wait_gives_up_and_the_handle_stays_usable(PVFinder, precision):
    from paper_2602_19959_gb300.pvf import PVF_ERR_TIMEOUT
    w = synth.he_weights(0)
    kw = {}
    if precision == "fp8":
        cal = synth.generate_standard(512, 1)
        pc = PVFinder(w, precision="bf16", max_events=512, max_pv_per_event=8)
        kw["fp8_act_scales"] = pc.calibrate(*to_cuda(cal))
        pc.close()
    ev = synth.generate_standard(16, 0)
    pv = PVFinder(w, precision=precision, max_events=16, max_pv_per_event=672, **kw)
    logit1, c1 = run(pv, ev)
    assert pv.device_status() == 0
    t0 = time.perf_counter()
    pv.test_wait_timeout(16, 2000)
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    assert pv.device_status() == PVF_ERR_TIMEOUT
    assert elapsed < 0.5                      # gave up after its 2 ms limit, not the 1 s one
    logit2, c2 = run(pv, ev)
    assert pv.device_status() == 0
    np.testing.assert_array_equal(logit2, logit1)
    np.testing.assert_array_equal(c2, c1)


def test_the_float32_form_has_no_tensor_core_waits(PVFinder):
    from paper_2602_19959_gb300.pvf import PvfError, PVF_ERR_UNSUPPORTED
    pv = PVFinder(synth.he_weights(0), precision="fp32", max_events=4)
    with pytest.raises(PvfError) as ei:
        pv.test_wait_timeout(4, 1000)
    assert ei.value.code == PVF_ERR_UNSUPPORTED

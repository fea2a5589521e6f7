"""pvf_histogram_static: the entry point for callers that cannot allocate device memory.

It runs steps 1-2 with its scratch in a fixed array inside libpvf.so. Its output must
match the pooled entry point (pvf_stage_histogram of an FP32 handle) within the
histogram tolerance of the other tests, on two calls in a row: the second with other
events, fewer of them and a bypassed event, so that nothing from the first call leaks.
Collected last, so a failure here leaves every other test already run."""

import ctypes

import numpy as np
import pytest

import synth
from paper_2602_19959_gb300 import pvf as P
from tests.helpers import to_cuda


def test_static_rejects_oversize_batches_on_the_host():
    from paper_2602_19959_gb300 import builder, weights
    builder.build()
    lib = P.load()
    blob = weights.pack_blob(synth.he_weights(0))
    buf = ctypes.create_string_buffer(blob, len(blob))
    tr = P.PvfTracks()
    for k in range(9):
        tr.f[k] = 0x10000
    tr.n_tracks = 10
    assert lib.pvf_histogram_static(buf, len(blob), ctypes.byref(tr), 0x10000, 4097, 0x10000,
                                    None, None) == P.PVF_ERR_INVALID_ARG
    assert lib.pvf_histogram_static(buf, 10, ctypes.byref(tr), 0x10000, 1, 0x10000,
                                    None, None) == P.PVF_ERR_WEIGHTS


@pytest.mark.gpu
def test_static_histogram_matches_pooled_entry_point_twice():
    import torch
    from paper_2602_19959_gb300 import build, PVFinder
    build()
    w = synth.he_weights(0, bias_std=0.05)
    pooled = PVFinder(w, precision="fp32", max_events=64, max_tracks_per_event=2048)
    calls = [synth.generate_standard(16, 0), synth.generate_standard(9, 7)]
    bad = calls[1]
    bad.offsets[3] = bad.offsets[2] - 1          # event 2 of the second call is bypassed
    for call, ev in enumerate(calls):
        feats, offs = to_cuda(ev)
        n = ev.n_events
        want = torch.zeros((n, 4000), dtype=torch.float32, device="cuda")
        pooled.stage_histogram(feats, offs, want)
        got = torch.full((n, 4000), -1.0, dtype=torch.float32, device="cuda")
        bypass = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        P.histogram_static(w, feats, offs, got, bypass)
        torch.cuda.synchronize()
        g, r, b = got.cpu().numpy(), want.cpu().numpy(), bypass.cpu().numpy()
        for e in range(n):
            scale = max(float(np.max(np.abs(r[e]))), 1e-30)
            assert np.max(np.abs(g[e] - r[e])) <= 1e-4 * scale, (call, e)
        expect = np.zeros(n, np.int32)
        if call == 1:
            expect[2] = 1
            assert np.all(g[2] == 0)
        np.testing.assert_array_equal(b, expect)

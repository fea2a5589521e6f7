"""CPU-only checks of the C-ABI library: it builds, loads, exports every symbol that
include/pvf.h declares, and rejects bad arguments on the host before any CUDA call."""

import ctypes
import os
import re
import struct

import numpy as np
import pytest

import synth
from paper_2602_19959_gb300 import builder, pvf as P, weights as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    builder.build()
    return P.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pvf.h")).read()
    return sorted(set(re.findall(r"PVF_API\s+[\w\s\*]+?\b(pvf_\w+)\s*\(", src)))


def test_header_declares_expected_api():
    syms = declared_symbols()
    for s in ("pvf_create", "pvf_infer", "pvf_destroy", "pvf_pool_bytes_required",
              "pvf_status_str", "pvf_last_device_status"):
        assert s in syms
    assert set(syms) == set(P.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_status_strings(lib):
    assert lib.pvf_status_str(0) == b"ok"
    assert b"pool" in lib.pvf_status_str(2)
    assert lib.pvf_status_str(12345)
    assert lib.pvf_version() >> 16 >= 1


def test_pool_bytes_required_and_config_validation(lib):
    fp32 = P.pool_bytes_required(precision="fp32", max_events=1000)
    bf16 = P.pool_bytes_required(precision="bf16", max_events=1000)
    fp8 = P.pool_bytes_required(precision="fp8", max_events=1000)
    fp16 = P.pool_bytes_required(precision="fp16", max_events=1000)
    assert fp32 > bf16 > fp8 > 0
    assert fp16 == bf16                              # same 16-bit activation layout
    assert fp32 < 2 * 1024 ** 3                      # the 1000-event plan fits a 2 GB pool
    chunked = P.pool_bytes_required(precision="fp32", max_events=1000, chunk_events=100)
    assert chunked < fp32 / 5
    assert P.pool_bytes_required(precision="bf16", max_events=1000, boundary_mm=0.5) == bf16
    # the wide UNet (base width 32): float32 only, twice the activation bytes
    fp32w = P.pool_bytes_required(precision="fp32", max_events=1000, unet_width=32)
    assert 1.9 * fp32 < fp32w < 2.1 * fp32
    assert P.pool_bytes_required(precision="fp32", max_events=1000, unet_width=16) == fp32
    for prec in ("bf16", "fp16", "fp8"):
        # the wide network and the per-interval layout exist in every form, not combined
        out = ctypes.c_size_t(0)
        for kw in (dict(unet_width=32), dict(per_interval=True)):
            cfg, _ = P.make_config(precision=prec, max_events=10, **kw)
            assert lib.pvf_pool_bytes_required(ctypes.byref(cfg), ctypes.byref(out)) == P.PVF_OK
        cfg, _ = P.make_config(precision=prec, max_events=10, unet_width=32, per_interval=True)
        assert lib.pvf_pool_bytes_required(ctypes.byref(cfg), ctypes.byref(out)) == P.PVF_ERR_UNSUPPORTED
    cfg, _ = P.make_config(precision="fp32", max_events=10, unet_width=32, per_interval=True)
    out = ctypes.c_size_t(0)
    assert lib.pvf_pool_bytes_required(ctypes.byref(cfg), ctypes.byref(out)) == P.PVF_ERR_UNSUPPORTED
    # a launch schedule changes grids only: the plan is the same
    sched = {"front": 1, "enc2": 3, "dec3_up2": 1, "tail": 4}
    assert P.pool_bytes_required(precision="bf16", max_events=1000, schedule=sched) == bf16
    # the per-interval layout: 40 sequences of 104 bins per event (e4: 17 rows x 128 channels)
    iv = P.pool_bytes_required(precision="fp32", max_events=1000, per_interval=True)
    assert 1.25 * fp32 < iv < 1.45 * fp32
    for bad in (dict(max_events=0), dict(max_tracks_per_event=0), dict(max_tracks_per_event=9000),
                dict(max_pv_per_event=0), dict(chunk_events=-1), dict(precision=7),
                dict(boundary_mm=-0.1), dict(boundary_mm=5.0), dict(boundary_mm=float("nan")),
                dict(unet_width=24), dict(unet_width=64), dict(unet_width=-16),
                dict(per_interval=2), dict(per_interval=-1), dict(schedule={"front": -1}),
                dict(schedule={"dec3_up2": -2}), dict(schedule={"tail": -1})):
        kw = dict(precision="fp32", max_events=10)
        kw.update(bad)
        cfg, _ = P.make_config(**kw)
        out = ctypes.c_size_t(0)
        assert lib.pvf_pool_bytes_required(ctypes.byref(cfg), ctypes.byref(out)) == P.PVF_ERR_INVALID_ARG


def test_create_rejects_bad_arguments_without_cuda(lib):
    cfg, _ = P.make_config(precision="fp32", max_events=4)
    h = ctypes.c_void_p()
    blob = W.pack_blob(synth.he_weights(0))
    buf = ctypes.create_string_buffer(blob, len(blob))
    # null pool, misaligned pool: rejected before any CUDA call
    assert lib.pvf_create(buf, len(blob), None, 1 << 30, ctypes.byref(cfg), None, ctypes.byref(h)) == 1
    assert lib.pvf_create(buf, len(blob), 0x1001, 1 << 30, ctypes.byref(cfg), None, ctypes.byref(h)) == 1
    # corrupted blob
    bad = bytearray(blob)
    bad[0:4] = b"XXXX"
    bbuf = ctypes.create_string_buffer(bytes(bad), len(bad))
    assert lib.pvf_create(bbuf, len(bad), 0x10000, 1 << 30, ctypes.byref(cfg), None, ctypes.byref(h)) == 3
    # truncated blob
    assert lib.pvf_create(buf, 100, 0x10000, 1 << 30, ctypes.byref(cfg), None, ctypes.byref(h)) == 3
    # pool too small
    assert lib.pvf_create(buf, len(blob), 0x10000, 1024, ctypes.byref(cfg), None, ctypes.byref(h)) == 2
    # non-finite weight
    wd = synth.he_weights(0)
    wd["dec3"][0][0, 0, 0] = np.nan
    nb = W.pack_blob(wd)
    nbuf = ctypes.create_string_buffer(nb, len(nb))
    assert lib.pvf_create(nbuf, len(nb), 0x10000, 1 << 30, ctypes.byref(cfg), None, ctypes.byref(h)) == 3
    # a width-32 blob under a width-16 config (and the reverse): ERR_WEIGHTS, before CUDA
    wide = W.pack_blob(synth.he_weights(0, c0=32))
    wbuf = ctypes.create_string_buffer(wide, len(wide))
    assert lib.pvf_create(wbuf, len(wide), 0x10000, 1 << 34, ctypes.byref(cfg), None, ctypes.byref(h)) == 3
    cfg32, _ = P.make_config(precision="fp32", max_events=4, unet_width=32)
    assert lib.pvf_create(buf, len(blob), 0x10000, 1 << 34, ctypes.byref(cfg32), None, ctypes.byref(h)) == 3
    # a valid blob of either width, in any order, parses: with a pool too small, create
    # stops at POOL_TOO_SMALL (after the blob checks, before any CUDA call)
    for b, c in ((buf, cfg), (wbuf, cfg32), (buf, cfg), (wbuf, cfg32)):
        assert lib.pvf_create(b, len(b.raw), 0x10000, 1024, ctypes.byref(c), None, ctypes.byref(h)) == 2
    # infer with a null handle
    assert lib.pvf_infer(None, None, None, 1, None, None, None) == 1
    assert lib.pvf_destroy(None) == 0


def test_blob_layout():
    blob = W.pack_blob(synth.he_weights(0))
    magic, ver, c0, hid, out, nl, r0, r1 = struct.unpack_from("<4s7I", blob, 0)
    assert (magic, ver, c0, hid, out, nl) == (b"PVFW", 1, 16, 32, 100, 17)
    name, ndim, s0, s1, s2, nb, _, wo, bo = struct.unpack_from("<8s6IQQ", blob, 32 + 48 * 11)
    assert name.rstrip(b"\0") == b"dec3" and (ndim, s0, s1, s2, nb) == (3, 64, 128, 5, 64)
    w = np.frombuffer(blob, dtype="<f4", count=64 * 128 * 5, offset=wo).reshape(64, 128, 5)
    np.testing.assert_array_equal(w, synth.he_weights(0)["dec3"][0])
    assert wo % 16 == 0 and bo % 16 == 0


def _serve_bytes(lib, max_pv=64, **kw):
    cfg = P.PvfServeConfig()
    cfg.max_batch, cfg.max_tracks_per_batch, cfg.max_inflight, cfg.min_batch = 32, 8000, 2, 1
    for k, v in kw.items():
        setattr(cfg, k, v)
    out = ctypes.c_size_t(0)
    return lib.pvf_serve_bytes_required(ctypes.byref(cfg), max_pv, ctypes.byref(out)), out.value


def test_serve_slot_sizing_and_validation(lib):
    """A serving slot of the copy form holds one batch: 9 feature rows of
    max_tracks_per_batch floats and max_batch + 1 offsets, then the counts, then
    max_batch x max_pv z values, each part 256-byte aligned; max_inflight slots in all."""
    align = lambda x: (x + 255) // 256 * 256
    slot = align(align(align(4 * 9 * 8000 + 4 * 33) + 4 * 32) + 4 * 32 * 64)
    st, n2 = _serve_bytes(lib)
    assert st == 0 and n2 == 2 * slot
    st, n5 = _serve_bytes(lib, max_inflight=5)
    assert st == 0 and n5 == 5 * slot
    for bad in (dict(max_batch=0), dict(max_inflight=0), dict(max_inflight=17),
                dict(max_tracks_per_batch=0)):
        assert _serve_bytes(lib, **bad)[0] == P.PVF_ERR_INVALID_ARG
    assert _serve_bytes(lib, max_pv=0)[0] == P.PVF_ERR_INVALID_ARG
    out = ctypes.c_size_t(0)
    assert lib.pvf_serve_bytes_required(None, 64, ctypes.byref(out)) == P.PVF_ERR_INVALID_ARG


def test_wait_timeout_test_hook_rejects_bad_arguments(lib):
    assert lib.pvf_test_wait_timeout(None, 1, 1000, None) == P.PVF_ERR_INVALID_ARG


def test_config_struct_layout():
    """The ctypes mirrors of the C structs keep the header's sizes and offsets."""
    assert ctypes.sizeof(P.PvfConfig) == 48 and P.PvfConfig.schedule.offset == 40
    assert ctypes.sizeof(P.PvfSchedule) == 32
    assert P.PvfConfig.boundary_mm.offset == 20 and P.PvfConfig.unet_width.offset == 24
    assert P.PvfConfig.per_interval.offset == 28 and P.PvfConfig.fp8_act_scales.offset == 32
    assert ctypes.sizeof(P.PvfServeConfig) == 32 and P.PvfServeConfig.flags.offset == 20
    assert P.PvfServeConfig.launch_lead_us.offset == 24

"""ctypes binding of libpvf (include/pvf.h): argument marshalling only.

Every step of the inference path runs in the library's CUDA kernels. PyTorch is used
for device memory (the fixed pool, inputs and outputs) and for the current stream;
tensors are passed as raw device pointers. If libpvf.so has not been built, loading
fails loudly: there is no fallback implementation.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .weights import pack_blob, unet_width

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpvf.so")

PVF_OK = 0
PVF_ERR_INVALID_ARG = 1
PVF_ERR_POOL_TOO_SMALL = 2
PVF_ERR_WEIGHTS = 3
PVF_ERR_CUDA = 4
PVF_ERR_TIMEOUT = 5
PVF_ERR_UNSUPPORTED = 6
PVF_WARN_EVENTS_SKIPPED = 16
PVF_WARN_TRUNCATED = 17

PRECISIONS = {"fp32": 0, "bf16": 1, "fp8": 2, "fp16": 3}
N_BINS = 4000
N_ACT_SCALES = 16

EXPORTED = ("pvf_pool_bytes_required", "pvf_create", "pvf_infer", "pvf_infer_ex",
            "pvf_stage_histogram", "pvf_stage_unet", "pvf_stage_peaks",
            "pvf_last_device_status", "pvf_profile_enable", "pvf_profile_read", "pvf_calibrate",
            "pvf_histogram_static", "pvf_graph_create", "pvf_graph_create_dynamic",
            "pvf_graph_launch", "pvf_graph_destroy",
            "pvf_serve_bytes_required", "pvf_serve_replay", "pvf_test_wait_timeout",
            "pvf_destroy", "pvf_status_str", "pvf_version")


class PvfSchedule(ctypes.Structure):
    _fields_ = [("front_ctas_per_sm", ctypes.c_int32), ("conv_ctas_per_sm", ctypes.c_int32 * 6),
                ("tail_ctas_per_sm", ctypes.c_int32)]

    CONV = ("enc2", "enc3", "enc4_up3", "dec3_up2", "dec2_up1", "dec1_final")

    @classmethod
    def from_dict(cls, d: dict):
        """{"front": n, "enc2": n, ..., "dec1_final": n, "tail": n} (missing keys: 0 = default)."""
        q = cls()
        q.front_ctas_per_sm = int(d.get("front", 0))
        q.tail_ctas_per_sm = int(d.get("tail", 0))
        for i, k in enumerate(cls.CONV):
            q.conv_ctas_per_sm[i] = int(d.get(k, 0))
        return q


class PvfConfig(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("max_events", ctypes.c_int32),
                ("max_tracks_per_event", ctypes.c_int32), ("max_pv_per_event", ctypes.c_int32),
                ("chunk_events", ctypes.c_int32), ("boundary_mm", ctypes.c_float),
                ("unet_width", ctypes.c_int32), ("per_interval", ctypes.c_int32),
                ("fp8_act_scales", ctypes.c_void_p), ("schedule", ctypes.c_void_p)]


class PvfTracks(ctypes.Structure):
    _fields_ = [("f", ctypes.c_void_p * 9), ("n_tracks", ctypes.c_int64)]


class PvfKernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int32), ("total_ms", ctypes.c_float)]


class PvfServeConfig(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("max_tracks_per_batch", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32), ("min_batch", ctypes.c_int32),
                ("max_wait_us", ctypes.c_float), ("flags", ctypes.c_int32),
                ("launch_lead_us", ctypes.c_float), ("reserved", ctypes.c_int32)]

SERVE_STREAM_LAUNCH = 1
SERVE_COPY = 2


class PvfError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_str(code)} ({code})")


_lock = threading.Lock()
_lib = None


def load(path: str = None):
    """Loads libpvf.so (LIB_PATH unless given) and declares the C signatures. Raises if it
    is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2602_19959_gb300.build()")
        lib = ctypes.CDLL(path)
        P, I32, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
        S = ctypes.c_int
        sig = {
            "pvf_pool_bytes_required": (S, [ctypes.POINTER(PvfConfig), ctypes.POINTER(SZ)]),
            "pvf_create": (S, [P, SZ, P, SZ, ctypes.POINTER(PvfConfig), P, ctypes.POINTER(P)]),
            "pvf_infer": (S, [P, ctypes.POINTER(PvfTracks), P, I32, P, P, P]),
            "pvf_infer_ex": (S, [P, ctypes.POINTER(PvfTracks), P, I32, P, P, P, P, P]),
            "pvf_stage_histogram": (S, [P, ctypes.POINTER(PvfTracks), P, I32, P, P]),
            "pvf_stage_unet": (S, [P, P, I32, P, P]),
            "pvf_stage_peaks": (S, [P, P, I32, P, P, P]),
            "pvf_last_device_status": (S, [P, ctypes.POINTER(I32), P]),
            "pvf_profile_enable": (S, [P, I32]),
            "pvf_profile_read": (S, [P, ctypes.POINTER(PvfKernelTime), I32, ctypes.POINTER(I32), P]),
            "pvf_calibrate": (S, [P, ctypes.POINTER(PvfTracks), P, I32, P, P]),
            "pvf_histogram_static": (S, [P, SZ, ctypes.POINTER(PvfTracks), P, I32, P, P, P]),
            "pvf_graph_create": (S, [P, ctypes.POINTER(PvfTracks), P, I32, P, P, ctypes.POINTER(P)]),
            "pvf_graph_create_dynamic": (S, [P, ctypes.POINTER(PvfTracks), P, P, I32, P, P,
                                             ctypes.POINTER(P)]),
            "pvf_graph_launch": (S, [P, P]),
            "pvf_graph_destroy": (S, [P]),
            "pvf_serve_bytes_required": (S, [ctypes.POINTER(PvfServeConfig), I32, ctypes.POINTER(SZ)]),
            "pvf_serve_replay": (S, [P, ctypes.POINTER(PvfServeConfig), ctypes.POINTER(P), P, I32, P, P,
                                     I32, P, SZ, P, P, P, P, P]),
            "pvf_test_wait_timeout": (S, [P, I32, ctypes.c_uint32, P]),
            "pvf_destroy": (S, [P]),
            "pvf_status_str": (ctypes.c_char_p, [S]),
            "pvf_version": (I32, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_str(code: int) -> str:
    try:
        return load().pvf_status_str(code).decode()
    except Exception:
        return "unknown"


def _check(code: int, where: str, allow_warn: bool = False):
    if code != PVF_OK and not (allow_warn and code >= PVF_WARN_EVENTS_SKIPPED):
        raise PvfError(code, where)
    return code


def make_config(precision="fp32", max_events=1, max_tracks_per_event=2048, max_pv_per_event=64,
                chunk_events=0, fp8_act_scales=None, boundary_mm=0.0, unet_width=0,
                per_interval=False, schedule=None):
    cfg = PvfConfig()
    cfg.boundary_mm = boundary_mm
    cfg.unet_width = unet_width
    cfg.per_interval = int(per_interval)
    cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    cfg.max_events = max_events
    cfg.max_tracks_per_event = max_tracks_per_event
    cfg.max_pv_per_event = max_pv_per_event
    cfg.chunk_events = chunk_events
    keep = []
    if fp8_act_scales is not None:
        scales = np.ascontiguousarray(fp8_act_scales, dtype=np.float32)
        keep.append(scales)
        cfg.fp8_act_scales = scales.ctypes.data
    if schedule is not None:
        q = schedule if isinstance(schedule, PvfSchedule) else PvfSchedule.from_dict(schedule)
        keep.append(q)
        cfg.schedule = ctypes.addressof(q)
    return cfg, keep


def pool_bytes_required(**cfg_kwargs) -> int:
    cfg, _ = make_config(**cfg_kwargs)
    out = ctypes.c_size_t(0)
    _check(load().pvf_pool_bytes_required(ctypes.byref(cfg), ctypes.byref(out)), "pvf_pool_bytes_required")
    return int(out.value)


def _stream_ptr(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def tracks_struct(features) -> PvfTracks:
    """features: CUDA float32 tensor [9, n_tracks] (rows contiguous) or a list of 9."""
    t = PvfTracks()
    rows = [features[k] for k in range(9)]
    t.n_tracks = int(rows[0].numel())
    for k, r in enumerate(rows):
        if not r.is_cuda or r.dtype.itemsize != 4 or not r.is_contiguous():
            raise ValueError("features must be contiguous CUDA float32 rows")
        if r.numel() != t.n_tracks:
            raise ValueError("all feature rows must have the same length")
        t.f[k] = r.data_ptr()
    return t


def _check_out(t, shape, itemsize, name):
    """An output tensor the kernels write: CUDA, contiguous, of this shape and element size."""
    if not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != tuple(shape) or \
            t.dtype.itemsize != itemsize or t.dtype.is_complex:
        raise ValueError(f"{name} must be a contiguous CUDA tensor of shape {tuple(shape)} "
                         f"and {itemsize}-byte elements")


def histogram_static(weights: dict, features, offsets, out_hist, out_bypass=None, stream=None):
    """Steps 1-2 through pvf_histogram_static (no device allocation by the library)."""
    lib = load()
    blob = pack_blob(weights)
    buf = ctypes.create_string_buffer(blob, len(blob))
    tr = tracks_struct(features)
    n = int(offsets.numel() - 1)
    _check_out(out_hist, (n, N_BINS), 4, "out_hist")
    if out_bypass is not None:
        _check_out(out_bypass, (n,), 4, "out_bypass")
    _check(lib.pvf_histogram_static(buf, len(blob), ctypes.byref(tr), offsets.data_ptr(), n,
                                    out_hist.data_ptr(),
                                    out_bypass.data_ptr() if out_bypass is not None else None,
                                    _stream_ptr(stream)), "pvf_histogram_static")
    return out_hist


class Graph:
    """A captured launch sequence; keeps the captured buffers alive."""

    def __init__(self, lib, handle, keep):
        self.lib, self.handle, self._keep = lib, handle, keep

    def launch(self, stream=None):
        _check(self.lib.pvf_graph_launch(self.handle, _stream_ptr(stream)), "pvf_graph_launch")

    def close(self):
        if self.handle:
            self.lib.pvf_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PVFinder:
    """Owns a pool tensor and a pvf_handle; every method maps to one C entry point.

    weights: {layer: (W, b)} in PyTorch layouts (the UNet base width, 16 or 32, is taken
    from enc1). precision: "fp32", "bf16", "fp16" or "fp8" (fp8 needs fp8_act_scales,
    e.g. from calibrate() of a bf16 instance). max_events / max_tracks_per_event /
    max_pv_per_event / chunk_events: the frozen plan of pvf_config. boundary_mm: width of
    the band in which a track also fills the neighbouring slice (0: none).
    per_interval: each interval runs the UNet as its own 104-bin sequence (width 16; with
    width 32 it raises PvfError with PVF_ERR_UNSUPPORTED). schedule: launch schedule (a dict of CTAs per SM per kernel
    family, e.g. the autotuner's table; None: the defaults)."""

    def __init__(self, weights: dict, precision="fp32", max_events=1024,
                 max_tracks_per_event=2048, max_pv_per_event=64, chunk_events=0,
                 fp8_act_scales=None, device=None, stream=None, boundary_mm=0.0,
                 per_interval=False, schedule=None):
        import torch
        self.lib = load()
        self.device = torch.device(device or "cuda")
        # the UNet base width follows the weights (the blob records it too)
        self.cfg, self._keep = make_config(precision, max_events, max_tracks_per_event,
                                           max_pv_per_event, chunk_events, fp8_act_scales,
                                           boundary_mm, unet_width(weights), per_interval,
                                           schedule)
        need = ctypes.c_size_t(0)
        _check(self.lib.pvf_pool_bytes_required(ctypes.byref(self.cfg), ctypes.byref(need)),
               "pvf_pool_bytes_required")
        self.pool_bytes = int(need.value)
        self.pool = torch.empty(self.pool_bytes, dtype=torch.uint8, device=self.device)
        blob = pack_blob(weights)
        self._blob = ctypes.create_string_buffer(blob, len(blob))
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(self.lib.pvf_create(self._blob, len(blob), self.pool.data_ptr(), self.pool_bytes,
                                       ctypes.byref(self.cfg), _stream_ptr(stream), ctypes.byref(h)),
                   "pvf_create")
        self.handle = h
        self.max_events = max_events
        self.max_pv = max_pv_per_event

    def close(self):
        if getattr(self, "handle", None):
            self.lib.pvf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def alloc_outputs(self, n_events: int):
        import torch
        z = torch.empty((n_events, self.max_pv), dtype=torch.float32, device=self.device)
        c = torch.empty((n_events,), dtype=torch.int32, device=self.device)
        return z, c

    def infer(self, features, offsets, n_events=None, out=None, hist=None, logit=None, stream=None):
        """features CUDA float32 [9, n_tracks]; offsets CUDA int32 [n_events + 1].
        Returns (pv_z [n, max_pv], pv_count [n]); enqueued on the current stream."""
        n = int(offsets.numel() - 1) if n_events is None else int(n_events)
        z, c = out if out is not None else self.alloc_outputs(n)
        tr = tracks_struct(features)
        _check(self.lib.pvf_infer_ex(self.handle, ctypes.byref(tr), offsets.data_ptr(), n,
                                     z.data_ptr(), c.data_ptr(),
                                     hist.data_ptr() if hist is not None else None,
                                     logit.data_ptr() if logit is not None else None,
                                     _stream_ptr(stream)), "pvf_infer_ex")
        return z, c

    def stage_histogram(self, features, offsets, out_hist, stream=None):
        tr = tracks_struct(features)
        n = int(offsets.numel() - 1)
        _check(self.lib.pvf_stage_histogram(self.handle, ctypes.byref(tr), offsets.data_ptr(), n,
                                            out_hist.data_ptr(), _stream_ptr(stream)),
               "pvf_stage_histogram")
        return out_hist

    def stage_unet(self, hist, out_logit, stream=None):
        n = int(hist.shape[0])
        _check(self.lib.pvf_stage_unet(self.handle, hist.data_ptr(), n, out_logit.data_ptr(),
                                       _stream_ptr(stream)), "pvf_stage_unet")
        return out_logit

    def stage_peaks(self, logit, out=None, stream=None):
        n = int(logit.shape[0])
        z, c = out if out is not None else self.alloc_outputs(n)
        _check(self.lib.pvf_stage_peaks(self.handle, logit.data_ptr(), n, z.data_ptr(), c.data_ptr(),
                                        _stream_ptr(stream)), "pvf_stage_peaks")
        return z, c

    def profile_enable(self, on: bool = True):
        _check(self.lib.pvf_profile_enable(self.handle, 1 if on else 0), "pvf_profile_enable")

    def profile_read(self, stream=None) -> dict:
        """{kernel family: (launches, total_ms)} since the last read (synchronises)."""
        buf = (PvfKernelTime * 64)()
        n = ctypes.c_int32(0)
        _check(self.lib.pvf_profile_read(self.handle, buf, 64, ctypes.byref(n), _stream_ptr(stream)),
               "pvf_profile_read")
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(n.value)}

    def calibrate(self, features, offsets, stream=None) -> np.ndarray:
        """FP8 activation scales from a calibration pass of this (bf16) handle."""
        tr = tracks_struct(features)
        n = int(offsets.numel() - 1)
        out = np.zeros(N_ACT_SCALES, dtype=np.float32)
        _check(self.lib.pvf_calibrate(self.handle, ctypes.byref(tr), offsets.data_ptr(), n,
                                      out.ctypes.data, _stream_ptr(stream)), "pvf_calibrate")
        return out

    def capture_graph(self, features, offsets, out):
        """A CUDA graph of the whole launch sequence for these fixed buffers."""
        tr = tracks_struct(features)
        n = int(offsets.numel() - 1)
        z, c = out
        g = ctypes.c_void_p()
        _check(self.lib.pvf_graph_create(self.handle, ctypes.byref(tr), offsets.data_ptr(), n,
                                         z.data_ptr(), c.data_ptr(), ctypes.byref(g)), "pvf_graph_create")
        return Graph(self.lib, g, (features, offsets, out))

    def capture_graph_dynamic(self, features, offsets, n_events, out):
        """A CUDA graph of the whole launch sequence for these fixed buffers that reads
        its event count from n_events (CUDA int32 tensor of one element) at each launch;
        out covers its capacity, offsets.numel() - 1 events."""
        tr = tracks_struct(features)
        n = int(offsets.numel() - 1)
        z, c = out
        g = ctypes.c_void_p()
        _check(self.lib.pvf_graph_create_dynamic(self.handle, ctypes.byref(tr), offsets.data_ptr(),
                                                 n_events.data_ptr(), n, z.data_ptr(), c.data_ptr(),
                                                 ctypes.byref(g)), "pvf_graph_create_dynamic")
        return Graph(self.lib, g, (features, offsets, n_events, out))

    def serve_replay(self, store, arrival_ns, request_event, max_batch=128,
                     max_tracks_per_batch=None, max_inflight=2, min_batch=1, max_wait_us=0.0,
                     want_z=False, graphs=True, copy=False, launch_lead_us=0.0, stream=None):
        """Continuous-batching replay (pvf_serve_replay). store: an EventBatch (host SoA).
        copy=True: the copy form (device slots and per-bucket graphs) instead of the
        gather form; graphs=False (copy form) enqueues pvf_infer per batch.
        launch_lead_us > 0: the next batch is admitted only once the running one is
        predicted to end within that many microseconds.
        Returns (done_ns int64 [n], pv_count int32 [n], batches, z [n, max_pv] or None)."""
        import torch
        feats = np.ascontiguousarray(store.features, dtype=np.float32)
        offs = np.ascontiguousarray(store.offsets, dtype=np.int32)
        arrival_ns = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        request_event = np.ascontiguousarray(request_event, dtype=np.int32)
        n = int(arrival_ns.shape[0])
        if max_tracks_per_batch is None:
            max_tracks_per_batch = int(max(np.diff(offs).max(), 1) * max_batch)
        cfg = PvfServeConfig(max_batch, max_tracks_per_batch, max_inflight, min_batch,
                             float(max_wait_us),
                             (0 if graphs else SERVE_STREAM_LAUNCH) | (SERVE_COPY if copy else 0),
                             float(launch_lead_us))
        need = ctypes.c_size_t(0)
        _check(self.lib.pvf_serve_bytes_required(ctypes.byref(cfg), self.max_pv, ctypes.byref(need)),
               "pvf_serve_bytes_required")
        slots = torch.empty(int(need.value), dtype=torch.uint8, device=self.device)
        fptr = (ctypes.c_void_p * 9)(*[feats[k].ctypes.data for k in range(9)])
        done = np.zeros(n, dtype=np.int64)
        cnt = np.zeros(n, dtype=np.int32)
        z = np.zeros((n, self.max_pv), dtype=np.float32) if want_z else None
        nb = ctypes.c_int32(0)
        _check(self.lib.pvf_serve_replay(self.handle, ctypes.byref(cfg), fptr, offs.ctypes.data,
                                         int(offs.shape[0] - 1), arrival_ns.ctypes.data,
                                         request_event.ctypes.data, n, slots.data_ptr(),
                                         int(need.value), done.ctypes.data, cnt.ctypes.data,
                                         z.ctypes.data if want_z else None,
                                         ctypes.byref(nb), _stream_ptr(stream)), "pvf_serve_replay")
        return done, cnt, int(nb.value), z

    def test_wait_timeout(self, n_events: int, limit_us: int, stream=None):
        """pvf_test_wait_timeout: a bounded wait that nothing completes (tests only)."""
        _check(self.lib.pvf_test_wait_timeout(self.handle, int(n_events), int(limit_us), _stream_ptr(stream)),
               "pvf_test_wait_timeout")

    def device_status(self, stream=None) -> int:
        v = ctypes.c_int32(0)
        _check(self.lib.pvf_last_device_status(self.handle, ctypes.byref(v), _stream_ptr(stream)),
               "pvf_last_device_status")
        return int(v.value)

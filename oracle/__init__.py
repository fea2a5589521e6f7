"""FP64 CPU oracle for PVFinder inference -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline and
reference legs) may import this package. The product path never calls it; the
oracle shares no code with the CUDA library and neither imports the other.

The arithmetic lives in ``pvf_oracle.c`` (plain C, double precision, direct loops,
following §2 of the paper step by step); this module compiles it with gcc into
``oracle/_build/liboracle.so`` on first use and wraps it with ctypes.

Parity status per function (pins live in tests/test_oracle_pins.py):
  slice_index        pinned: hand-computed boundary cases
  fc_track           pinned: numpy float64 matmul chain, zero-weight closed form
  event_histogram    pinned: closed form with constant FC output, permutation invariance
  conv1d_k5          pinned: numpy.convolve, delta kernel, linearity
  convT_k2s2         pinned: numpy.kron/einsum restatement, delta kernel
  maxpool2           pinned: numpy reshape-max
  unet               pinned: identity-UNet closed form, translation equivariance,
                     a second numpy statement on a short sequence
  peaks              pinned: hand-built histograms with known answers
  infer              whole-pipeline composition with random He weights: parity unpinned
                     beyond the stage pins and the second numpy statement
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pvf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NBINS = 4000
Z_LO = -100.0
BIN_W = 0.1
THRESHOLD = 0.01

ACT_NAMES = ("e1", "p1", "e2", "p2", "e3", "p3", "e4", "u3", "d3", "u2", "d2", "u1", "d1",
             "f", "prob")


def build(force: bool = False) -> str:
    """Compiles pvf_oracle.c into oracle/_build/liboracle.so (gcc, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
           "-fno-fast-math", "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OracleWeights(ctypes.Structure):
    _fields_ = [("c0", ctypes.c_int), ("fc_hidden", ctypes.c_int), ("fc_out", ctypes.c_int),
                ("fc_w", ctypes.c_void_p * 6), ("fc_b", ctypes.c_void_p * 6),
                ("enc_w", ctypes.c_void_p * 4), ("enc_b", ctypes.c_void_p * 4),
                ("up_w", ctypes.c_void_p * 3), ("up_b", ctypes.c_void_p * 3),
                ("dec_w", ctypes.c_void_p * 3), ("dec_b", ctypes.c_void_p * 3),
                ("fin_w", ctypes.c_void_p), ("fin_b", ctypes.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        lib.oracle_slice_index.argtypes = [ctypes.c_float]
        lib.oracle_slice_index.restype = I
        lib.oracle_fc_track.argtypes = [ctypes.POINTER(OracleWeights), P, P]
        lib.oracle_fc_track.restype = None
        lib.oracle_second_slice.argtypes = [ctypes.c_float, I, ctypes.c_float]
        lib.oracle_second_slice.restype = I
        lib.oracle_event_histogram.argtypes = [P, ctypes.c_int64, ctypes.c_int64,
                                               ctypes.POINTER(OracleWeights), ctypes.c_float, P]
        lib.oracle_event_histogram.restype = I
        lib.oracle_conv1d_k5.argtypes = [P, I, I, P, P, I, P]
        lib.oracle_conv1d_k5.restype = None
        lib.oracle_convT_k2s2.argtypes = [P, I, I, P, P, I, P]
        lib.oracle_convT_k2s2.restype = None
        lib.oracle_maxpool2.argtypes = [P, I, I, P]
        lib.oracle_maxpool2.restype = None
        lib.oracle_unet.argtypes = [ctypes.POINTER(OracleWeights), P, I, P, P, P]
        lib.oracle_unet.restype = I
        lib.oracle_peaks.argtypes = [P, P, I, ctypes.c_double, I, I, ctypes.c_double,
                                     ctypes.c_double, I, P, P]
        lib.oracle_peaks.restype = I
        lib.oracle_infer.argtypes = [P, P, ctypes.c_int64, I, I, ctypes.POINTER(OracleWeights),
                                     P, P, P, P, P, P, I, ctypes.c_double, ctypes.c_float, I, I]
        lib.oracle_unet_intervals.argtypes = [ctypes.POINTER(OracleWeights), P, P, P]
        lib.oracle_unet_intervals.restype = I
        lib.oracle_infer.restype = I
        _lib = lib
        return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Weights:
    """Float64 copies of {name: (W, b)} kept alive next to the ctypes struct."""

    def __init__(self, wdict: dict):
        self.arrays = {k: (_f64(w), _f64(b)) for k, (w, b) in wdict.items()}
        a = self.arrays
        s = OracleWeights()
        s.c0 = int(a["enc1"][0].shape[0])
        s.fc_hidden = int(a["fc1"][0].shape[0])
        s.fc_out = int(a["fc6"][0].shape[0])
        for i in range(6):
            s.fc_w[i] = a[f"fc{i + 1}"][0].ctypes.data
            s.fc_b[i] = a[f"fc{i + 1}"][1].ctypes.data
        for i in range(4):
            s.enc_w[i] = a[f"enc{i + 1}"][0].ctypes.data
            s.enc_b[i] = a[f"enc{i + 1}"][1].ctypes.data
        for i, lvl in enumerate((3, 2, 1)):
            s.up_w[i] = a[f"up{lvl}"][0].ctypes.data
            s.up_b[i] = a[f"up{lvl}"][1].ctypes.data
            s.dec_w[i] = a[f"dec{lvl}"][0].ctypes.data
            s.dec_b[i] = a[f"dec{lvl}"][1].ctypes.data
        s.fin_w = a["final"][0].ctypes.data
        s.fin_b = a["final"][1].ctypes.data
        self.struct = s


def _as_weights(w) -> Weights:
    return w if isinstance(w, Weights) else Weights(w)


def slice_index(z) -> np.ndarray:
    lib = _load()
    z = np.atleast_1d(np.asarray(z, dtype=np.float32))
    return np.array([lib.oracle_slice_index(ctypes.c_float(float(v))) for v in z], dtype=np.int32)


def fc_track(weights, x) -> np.ndarray:
    """FC net on one 9-vector (feature 2 already slice-relative)."""
    lib = _load()
    w = _as_weights(weights)
    x = _f64(x)
    out = np.zeros(w.struct.fc_out, dtype=np.float64)
    lib.oracle_fc_track(ctypes.byref(w.struct), _ptr(x), _ptr(out))
    return out


def _feature_ptrs(features: np.ndarray):
    features = np.ascontiguousarray(features, dtype=np.float32)
    ptrs = (ctypes.c_void_p * 9)(*[features[k].ctypes.data for k in range(9)])
    return features, ptrs


def second_slice(z, s, edge_mm) -> int:
    """Second slice of a boundary track of slice s at float32 z (-1: none)."""
    return _load().oracle_second_slice(ctypes.c_float(float(z)), int(s), ctypes.c_float(float(edge_mm)))


def event_histogram(weights, features: np.ndarray, edge_mm: float = 0.0):
    """Histogram [4000] of one event given float32 features [9, n]; returns (hist, dropped).
    edge_mm > 0 also adds boundary tracks to their second slice."""
    lib = _load()
    w = _as_weights(weights)
    features, ptrs = _feature_ptrs(features)
    hist = np.zeros(NBINS, dtype=np.float64)
    dropped = lib.oracle_event_histogram(ptrs, 0, features.shape[1], ctypes.byref(w.struct),
                                         ctypes.c_float(edge_mm), _ptr(hist))
    return hist, dropped


def conv1d_k5(x, W, b) -> np.ndarray:
    lib = _load()
    x, W, b = _f64(x), _f64(W), _f64(b)
    cin, L = x.shape
    cout = W.shape[0]
    assert W.shape == (cout, cin, 5) and b.shape == (cout,)
    y = np.zeros((cout, L), dtype=np.float64)
    lib.oracle_conv1d_k5(_ptr(x), cin, L, _ptr(W), _ptr(b), cout, _ptr(y))
    return y


def convT_k2s2(x, W, b) -> np.ndarray:
    lib = _load()
    x, W, b = _f64(x), _f64(W), _f64(b)
    cin, L = x.shape
    cout = W.shape[1]
    assert W.shape == (cin, cout, 2) and b.shape == (cout,)
    y = np.zeros((cout, 2 * L), dtype=np.float64)
    lib.oracle_convT_k2s2(_ptr(x), cin, L, _ptr(W), _ptr(b), cout, _ptr(y))
    return y


def maxpool2(x) -> np.ndarray:
    lib = _load()
    x = _f64(x)
    C, L = x.shape
    y = np.zeros((C, L // 2), dtype=np.float64)
    lib.oracle_maxpool2(_ptr(x), C, L, _ptr(y))
    return y


def unet(weights, hist, return_acts: bool = False):
    """(logit, prob) = UNet(hist) for one event; hist [L] with L divisible by 8.
    With return_acts, also a dict of every intermediate ([C][L] arrays)."""
    lib = _load()
    w = _as_weights(weights)
    hist = _f64(hist).reshape(-1)
    L = hist.shape[0]
    logit = np.zeros(L, dtype=np.float64)
    prob = np.zeros(L, dtype=np.float64)
    acts = None
    acts_arg = None
    if return_acts:
        c1 = w.struct.c0
        shapes = {"e1": (c1, L), "p1": (c1, L // 2), "e2": (2 * c1, L // 2),
                  "p2": (2 * c1, L // 4), "e3": (4 * c1, L // 4), "p3": (4 * c1, L // 8),
                  "e4": (8 * c1, L // 8), "u3": (4 * c1, L // 4), "d3": (4 * c1, L // 4),
                  "u2": (2 * c1, L // 2), "d2": (2 * c1, L // 2), "u1": (c1, L),
                  "d1": (c1, L), "f": (L,), "prob": (L,)}
        acts = {k: np.zeros(shapes[k], dtype=np.float64) for k in ACT_NAMES}
        acts_arg = (ctypes.c_void_p * len(ACT_NAMES))(*[acts[k].ctypes.data for k in ACT_NAMES])
    rc = lib.oracle_unet(ctypes.byref(w.struct), _ptr(hist), L, _ptr(logit), _ptr(prob), acts_arg)
    if rc != 0:
        raise RuntimeError(f"oracle_unet failed ({rc})")
    return (logit, prob, acts) if return_acts else (logit, prob)


def unet_intervals(weights, hist):
    """(logit, prob) [4000] of one event in the per-interval layout."""
    lib = _load()
    w = _as_weights(weights)
    hist = _f64(hist).reshape(-1)
    assert hist.shape[0] == NBINS
    logit = np.zeros(NBINS, dtype=np.float64)
    prob = np.zeros(NBINS, dtype=np.float64)
    if lib.oracle_unet_intervals(ctypes.byref(w.struct), _ptr(hist), _ptr(logit), _ptr(prob)) != 0:
        raise RuntimeError("oracle_unet_intervals failed")
    return logit, prob


def threshold_logit(thr: float = THRESHOLD) -> float:
    """The probability threshold thr expressed on the logit: ln(thr / (1 - thr))."""
    return float(np.log(thr / (1.0 - thr)))


def peaks(logit, prob=None, thr: float = THRESHOLD, hw: int = 5, hc: int = 3,
          z_lo: float = Z_LO, bw: float = BIN_W, max_pv: int = 1024):
    """Peak finder on one event. Decisions use the logits (prob = sigmoid(logit) when
    not given); centroid weights use prob. Returns (count, z[:k], bins[:k]), k =
    min(count, max_pv)."""
    lib = _load()
    f = _f64(logit).reshape(-1)
    if prob is None:
        with np.errstate(over="ignore"):
            prob = 1.0 / (1.0 + np.exp(-f))
    p = _f64(prob).reshape(-1)
    z = np.zeros(max(max_pv, 1), dtype=np.float64)
    bins = np.zeros(max(max_pv, 1), dtype=np.int32)
    n = lib.oracle_peaks(_ptr(f), _ptr(p), f.shape[0], threshold_logit(thr), hw, hc, z_lo, bw,
                         max_pv, _ptr(z), _ptr(bins))
    k = min(n, max_pv)
    return n, z[:k].copy(), bins[:k].copy()


def infer(weights, features: np.ndarray, offsets: np.ndarray, max_pv: int = 64,
          max_tracks_per_event: int = 1 << 30, want_hist: bool = False,
          want_logit: bool = False, want_prob: bool = False, nthreads: int = 1,
          thr: float = THRESHOLD, edge_mm: float = 0.0, per_interval: bool = False):
    """Whole-pipeline oracle over a batch. Returns a dict with pv_z [n, max_pv],
    pv_count [n] (-1 = bypassed event), n_dropped [n], and optionally hist / logit /
    prob ([n, 4000] each). edge_mm: boundary-track width (0 = none). per_interval: the
    UNet runs on each of the 40 intervals as its own 104-bin sequence."""
    lib = _load()
    w = _as_weights(weights)
    features, ptrs = _feature_ptrs(features)
    offsets = np.ascontiguousarray(offsets, dtype=np.int32)
    n = offsets.shape[0] - 1
    pv_z = np.full((max(n, 0), max_pv), np.nan, dtype=np.float64)
    pv_count = np.zeros(max(n, 0), dtype=np.int32)
    n_drop = np.zeros(max(n, 0), dtype=np.int32)
    hist = np.zeros((n, NBINS), dtype=np.float64) if want_hist else None
    logit = np.zeros((n, NBINS), dtype=np.float64) if want_logit else None
    prob = np.zeros((n, NBINS), dtype=np.float64) if want_prob else None
    rc = lib.oracle_infer(ptrs, _ptr(offsets), features.shape[1], n, max_tracks_per_event,
                          ctypes.byref(w.struct), _ptr(hist), _ptr(logit), _ptr(prob), _ptr(pv_z),
                          _ptr(pv_count), _ptr(n_drop), max_pv, thr, ctypes.c_float(edge_mm),
                          int(per_interval), nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle_infer failed ({rc})")
    out = {"pv_z": pv_z, "pv_count": pv_count, "n_dropped": n_drop}
    if want_hist:
        out["hist"] = hist
    if want_logit:
        out["logit"] = logit
    if want_prob:
        out["prob"] = prob
    return out

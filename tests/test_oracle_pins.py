"""Pins for the FP64 oracle: each stage checked against something other than itself.

Closed forms, PyTorch/numpy float64 library routines, exact rational arithmetic,
hand-built cases with hand-derived answers (tests/golden/peaks_handbuilt.json), and
invariants (permutation invariance of the histogram, translation equivariance of the
UNet). The cases are chosen so that a dropped term, a wrong sign or index, a
transposed operand or a swapped concat order fails at least one of them.
"""

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
import synth
from tests import ref_torch64 as ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_weights(seed=1, bias_std=0.3, c0=16):
    return synth.he_weights(seed=seed, bias_std=bias_std, c0=c0)


# ----------------------------------------------------------------- slice index

def exact_slice(z32: np.float32):
    """floor((z + 100) / 10) in exact rational arithmetic (no rounding)."""
    q = (Fraction(float(z32)) + 100) / 10
    return math.floor(q)


def test_slice_index_hand_cases():
    # slice s covers [-100 + 10 s, -90 + 10 s): boundaries belong to the upper slice
    cases = {-100.0: 0, -90.0: 1, -60.0: 4, 0.0: 10, 289.99: 38, 290.0: 39,
             299.99998: 39, 300.0: -1, -100.00001: -1, 1e30: -1, -1e30: -1,
             float("nan"): -1, float("inf"): -1, float("-inf"): -1}
    for z, s in cases.items():
        assert oracle.slice_index(z)[0] == s, z


def test_slice_index_matches_exact_floor_away_from_edges():
    rng = np.random.default_rng(5)
    z = rng.uniform(-100, 300, 20000).astype(np.float32)
    got = oracle.slice_index(z)
    for zi, si in zip(z, got):
        e = exact_slice(zi)
        # float32 rounding may only move a track that sits within a few ulps of an edge
        edge = -100 + 10 * round((float(zi) + 100) / 10)
        if abs(float(zi) - edge) > 1e-4:
            assert si == e, (zi, si, e)


def test_slice_index_one_ulp_around_edges():
    for s_edge in range(1, 40):
        z_edge = np.float32(-100 + 10 * s_edge)
        below = np.nextafter(z_edge, np.float32(-1e9))
        above = np.nextafter(z_edge, np.float32(1e9))
        assert oracle.slice_index(z_edge)[0] == s_edge
        assert oracle.slice_index(above)[0] == s_edge
        # one ulp below the edge: the exact quotient is below s_edge; float32 rounding of
        # (z + 100) / 10 may round up to s_edge, never to anything else
        assert oracle.slice_index(below)[0] in (s_edge - 1, s_edge)


# ----------------------------------------------------------------- FC network

def test_fc_matches_torch_float64():
    w = rand_weights(3, 0.2)
    rng = np.random.default_rng(7)
    for _ in range(5):
        x = rng.normal(0, 2, 9)
        got = oracle.fc_track(w, x)
        want = ref.fc_net(w, torch.as_tensor(x).reshape(1, 9)).numpy()[0]
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def test_fc_zero_weights_closed_form():
    w = rand_weights(3, 0.0)
    b6 = np.linspace(-30, 30, 100).astype(np.float32)
    w = {k: (np.zeros_like(W), np.zeros_like(b)) for k, (W, b) in w.items()}
    w["fc6"] = (w["fc6"][0], b6)
    got = oracle.fc_track(w, np.ones(9))
    # softplus(b) = log(1 + e^b) via numpy's logaddexp(0, b); above 20 the oracle returns b
    want = np.where(b6 > 20, b6.astype(np.float64), np.logaddexp(0.0, b6.astype(np.float64)))
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=0)
    assert np.max(np.abs(want - np.logaddexp(0.0, b6.astype(np.float64)))) < 3e-9


def test_fc_leaky_slope_single_path():
    # one unit carries x0 through five LeakyReLUs into every output: x0 = -2 gives
    # -2 * 0.01^5 before the softplus
    shapes = synth.layer_shapes()
    w = {k: (np.zeros(s[0], np.float32), np.zeros(s[1], np.float32)) for k, s in shapes.items()}
    for name in ("fc1", "fc2", "fc3", "fc4", "fc5"):
        w[name][0][0, 0] = 1.0
    w["fc6"][0][:, 0] = 1.0
    x = np.zeros(9)
    x[0] = -2.0
    got = oracle.fc_track(w, x)
    np.testing.assert_allclose(got, np.logaddexp(0.0, -2.0 * 0.01 ** 5), rtol=1e-15)
    x[0] = 3.0
    np.testing.assert_allclose(oracle.fc_track(w, x), np.logaddexp(0.0, 3.0), rtol=1e-15)


# ----------------------------------------------------------------- histogram

def test_histogram_closed_form_constant_fc():
    shapes = synth.layer_shapes()
    w = {k: (np.zeros(s[0], np.float32), np.zeros(s[1], np.float32)) for k, s in shapes.items()}
    b6 = np.linspace(-3, 3, 100).astype(np.float32)
    w["fc6"] = (w["fc6"][0], b6)
    ev = synth.generate_standard(3, 11)
    feats = ev.features[:, ev.offsets[1]:ev.offsets[2]]
    hist, dropped = oracle.event_histogram(w, feats)
    counts = np.zeros(40)
    for z in feats[2]:
        counts[exact_slice(z)] += 1   # generated z are never within ulps of an edge
    want = (counts[:, None] * np.logaddexp(0.0, b6.astype(np.float64))[None, :]).reshape(-1)
    np.testing.assert_allclose(hist, want, rtol=1e-13, atol=0)
    assert dropped == 0


def test_histogram_matches_torch_and_is_permutation_invariant():
    w = rand_weights(4, 0.1)
    ev = synth.generate_standard(4, 12)
    for e in range(4):
        feats = ev.features[:, ev.offsets[e]:ev.offsets[e + 1]]
        hist, _ = oracle.event_histogram(w, feats)
        np.testing.assert_allclose(hist, ref.histogram(w, feats), rtol=1e-12, atol=1e-12)
        perm = np.random.default_rng(e).permutation(feats.shape[1])
        hist2, _ = oracle.event_histogram(w, feats[:, perm])
        np.testing.assert_allclose(hist2, hist, rtol=1e-12, atol=1e-12)


def test_histogram_slice_relative_z_feature():
    # two tracks with the same position inside different slices give the same 100-bin
    # profile, shifted by one slice; a dropped or absolute z would break this
    w = rand_weights(6, 0.1)
    f = np.zeros((9, 1), np.float32)
    f[2, 0] = -95.0           # slice 0, z_rel = 5
    h0, _ = oracle.event_histogram(w, f)
    f[2, 0] = -85.0           # slice 1, z_rel = 5
    h1, _ = oracle.event_histogram(w, f)
    assert np.all(h0[100:] == 0) and np.all(h1[:100] == 0) and np.all(h1[200:] == 0)
    np.testing.assert_array_equal(h0[:100], h1[100:200])
    x = np.zeros(9)
    x[2] = 5.0
    np.testing.assert_allclose(h0[:100], oracle.fc_track(w, x), rtol=0, atol=0)


# ----------------------------------------------------------------- boundary tracks (§3)
# A track whose slice-relative z (float32) is below the width w also belongs to the slice
# below; one at or above 10 - w also to the slice above; never outside slices 0..39.

def _f32_below(x):
    return float(np.nextafter(np.float32(x), np.float32(-1e9)))


def test_second_slice_rule_hand_cases():
    w = 0.5
    cases = [(-89.5, 1, -1),                 # zr = 0.5: not below w
             (_f32_below(-89.5), 1, 0),      # zr one ulp below 0.5
             (-80.5, 1, 2),                  # zr = 9.5 = 10 - w: belongs above too
             (_f32_below(-80.5), 1, -1),     # just below 10 - w
             (-85.0, 1, -1),                 # middle of the slice
             (-99.8, 0, -1),                 # no slice below 0
             (299.7, 39, -1),                # no slice above 39
             (290.2, 39, 38),
             (-90.0, 1, 0)]                  # on the edge itself: zr = 0
    for z, s, want in cases:
        assert oracle.slice_index(z)[0] == s, z
        assert oracle.second_slice(z, s, w) == want, (z, s)
        assert oracle.second_slice(z, s, 0.0) == -1


def test_boundary_histogram_closed_form_constant_fc():
    """All FC weights zero: every evaluation gives softplus(b6) per bin, so each slice holds
    (number of tracks counted in it) x softplus(b6); counts derived by hand, w = 1 mm."""
    shapes = synth.layer_shapes()
    wts = {k: (np.zeros(s[0], np.float32), np.zeros(s[1], np.float32)) for k, s in shapes.items()}
    b6 = np.linspace(-3, 3, 100).astype(np.float32)
    wts["fc6"] = (wts["fc6"][0], b6)
    z = [-95.0,      # slice 0 only
         -90.5,      # slice 0, zr 9.5 >= 9: and slice 1
         -89.7,      # slice 1, zr 0.3 < 1: and slice 0
         -85.0,      # slice 1 only
         -99.5,      # slice 0, zr 0.5 < 1, but no slice below 0
         299.5,      # slice 39, zr 9.5, but no slice above 39
         150.2]      # slice 25, zr 0.2: and slice 24
    f = np.zeros((9, len(z)), np.float32)
    f[2] = z
    hist, dropped = oracle.event_histogram(wts, f, edge_mm=1.0)
    counts = np.zeros(40)
    counts[0], counts[1], counts[39], counts[25], counts[24] = 4, 3, 1, 1, 1
    want = (counts[:, None] * np.logaddexp(0.0, b6.astype(np.float64))[None, :]).reshape(-1)
    np.testing.assert_allclose(hist, want, rtol=1e-13, atol=0)
    assert dropped == 0
    plain, _ = oracle.event_histogram(wts, f, edge_mm=0.0)
    counts0 = np.zeros(40)
    counts0[0], counts0[1], counts0[39], counts0[25] = 3, 2, 1, 1
    np.testing.assert_allclose(plain, (counts0[:, None] * np.logaddexp(0.0, b6.astype(np.float64))).reshape(-1),
                               rtol=1e-13, atol=0)


def test_boundary_second_evaluation_uses_the_second_slice_offset():
    """With random weights, a boundary track adds to its second slice the FC output for
    the position relative to that slice (PyTorch float64 statement of the net), and its
    own slice's bins are those of the plain histogram."""
    wts = rand_weights(8, 0.2)
    rng = np.random.default_rng(9)
    for z, s, s2 in [(-79.7, 2, 1), (-60.4, 3, 4), (-89.9, 1, 0), (120.3, 22, 21)]:
        f = rng.normal(0, 0.1, (9, 1)).astype(np.float32)
        f[2, 0] = z
        hist, _ = oracle.event_histogram(wts, f, edge_mm=0.5)
        plain, _ = oracle.event_histogram(wts, f)
        x = f[:, 0].astype(np.float64)
        x[2] = float(np.float32(z)) - (-100.0 + 10.0 * s2)
        want2 = ref.fc_net(wts, torch.as_tensor(x).reshape(1, 9)).numpy()[0]
        np.testing.assert_allclose(hist[100 * s2:100 * s2 + 100], want2, rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(hist[100 * s:100 * s + 100], plain[100 * s:100 * s + 100])
        others = np.ones(40, bool)
        others[[s, s2]] = False
        assert np.all(hist.reshape(40, 100)[others] == 0)
        assert (x[2] < 0) == (s2 > s) and abs(x[2] - 5) > 5   # just outside [0, 10)


def test_boundary_infer_reduces_to_plain_at_zero_width():
    wts = rand_weights(2, 0.1)
    ev = synth.generate_standard(3, 4)
    a = oracle.infer(wts, ev.features, ev.offsets, want_hist=True)
    b = oracle.infer(wts, ev.features, ev.offsets, want_hist=True, edge_mm=0.0)
    c = oracle.infer(wts, ev.features, ev.offsets, want_hist=True, edge_mm=0.5)
    np.testing.assert_array_equal(a["hist"], b["hist"])
    assert np.all(c["hist"].sum(axis=1) > a["hist"].sum(axis=1))   # softplus > 0: more terms
    with pytest.raises(RuntimeError):
        oracle.infer(wts, ev.features, ev.offsets, edge_mm=5.0)


def test_histogram_drops_invalid_tracks():
    w = rand_weights(6, 0.1)
    f = np.zeros((9, 5), np.float32)
    f[2] = [-100.5, 300.0, 10.0, 20.0, 30.0]
    f[4, 3] = np.nan
    f[7, 4] = np.inf
    hist, dropped = oracle.event_histogram(w, f)
    assert dropped == 4
    only, _ = oracle.event_histogram(w, f[:, 2:3])
    np.testing.assert_array_equal(hist, only)


# ----------------------------------------------------------------- conv pieces

def test_conv1d_matches_numpy_convolve_and_torch():
    rng = np.random.default_rng(8)
    cin, cout, L = 3, 4, 17
    x = rng.normal(size=(cin, L))
    W = rng.normal(size=(cout, cin, 5))
    b = rng.normal(size=cout)
    got = oracle.conv1d_k5(x, W, b)
    want = np.zeros((cout, L))
    for co in range(cout):
        want[co] = b[co]
        for ci in range(cin):
            want[co] += np.convolve(x[ci], W[co, ci, ::-1], mode="same")
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)
    tw = F.conv1d(torch.as_tensor(x)[None], torch.as_tensor(W), torch.as_tensor(b), padding=2)
    np.testing.assert_allclose(got, tw[0].numpy(), rtol=1e-13, atol=1e-13)


def test_conv1d_delta_kernel_is_identity_and_linear():
    rng = np.random.default_rng(9)
    C, L = 5, 32
    x = rng.normal(size=(C, L))
    W = np.zeros((C, C, 5))
    for c in range(C):
        W[c, c, 2] = 1.0
    np.testing.assert_array_equal(oracle.conv1d_k5(x, W, np.zeros(C)), x)
    # shifted delta: tap 4 reads x[i + 2]
    W2 = np.zeros((C, C, 5))
    for c in range(C):
        W2[c, c, 4] = 1.0
    y = oracle.conv1d_k5(x, W2, np.zeros(C))
    np.testing.assert_array_equal(y[:, :-2], x[:, 2:])
    np.testing.assert_array_equal(y[:, -2:], 0)
    Wr = rng.normal(size=(3, C, 5))
    y1 = rng.normal(size=(C, L))
    a, bb = 1.7, -0.4
    lhs = oracle.conv1d_k5(a * x + bb * y1, Wr, np.zeros(3))
    rhs = a * oracle.conv1d_k5(x, Wr, np.zeros(3)) + bb * oracle.conv1d_k5(y1, Wr, np.zeros(3))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_convT_matches_torch_and_delta():
    rng = np.random.default_rng(10)
    cin, cout, L = 6, 3, 9
    x = rng.normal(size=(cin, L))
    W = rng.normal(size=(cin, cout, 2))
    b = rng.normal(size=cout)
    got = oracle.convT_k2s2(x, W, b)
    want = F.conv_transpose1d(torch.as_tensor(x)[None], torch.as_tensor(W), torch.as_tensor(b),
                              stride=2)[0].numpy()
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)
    # delta: channel c copied into both phases r = 0, 1 (nearest-neighbour upsampling)
    Wd = np.zeros((3, 3, 2))
    for c in range(3):
        Wd[c, c, :] = 1.0
    xd = rng.normal(size=(3, 8))
    np.testing.assert_array_equal(oracle.convT_k2s2(xd, Wd, np.zeros(3)), np.repeat(xd, 2, axis=1))


def test_maxpool_matches_torch():
    x = np.random.default_rng(11).normal(size=(4, 22))
    want = F.max_pool1d(torch.as_tensor(x)[None], 2)[0].numpy()
    np.testing.assert_array_equal(oracle.maxpool2(x), want)


# ----------------------------------------------------------------- UNet

@pytest.mark.parametrize("c0", [16, 32])
def test_unet_matches_torch_statement_short_sequence(c0):
    w = rand_weights(12, 0.2, c0=c0)
    x = np.abs(np.random.default_rng(13).normal(0, 5, 256))
    f, p, acts = oracle.unet(w, x, return_acts=True)
    f2, p2 = ref.unet(w, x)
    np.testing.assert_allclose(f, f2, rtol=1e-11, atol=1e-10)
    np.testing.assert_allclose(p, p2, rtol=1e-12, atol=1e-14)
    assert acts["e4"].shape == (8 * c0, 32) and acts["d1"].shape == (c0, 256)


def identity_unet_weights(a=0.5, c=-1.0, c0=16):
    """enc1 = delta on channel 0; dec1 = delta on the skip half's channel 0 with every
    upsampled-path weight 0; final = a * delta + c; everything else 0."""
    shapes = synth.layer_shapes(c0)
    w = {k: (np.zeros(s[0], np.float64), np.zeros(s[1], np.float64)) for k, s in shapes.items()}
    w["enc1"][0][0, 0, 2] = 1.0
    w["dec1"][0][0, c0 + 0, 2] = 1.0        # concat order [upsampled (0..c0-1), skip (c0..2c0-1)]
    w["final"][0][0, 0, 2] = a
    w["final"][1][0] = c
    return w


@pytest.mark.parametrize("c0", [16, 32])
def test_unet_identity_closed_form(c0):
    a, c = 0.5, -1.0
    w = identity_unet_weights(a, c, c0)
    h = np.random.default_rng(14).normal(0, 3, 4000)
    f, p = oracle.unet(w, h)
    lr = np.where(h > 0, h, 0.01 * h)
    lr2 = np.where(lr > 0, lr, 0.01 * lr)     # LeakyReLU after enc1 and after dec1
    np.testing.assert_allclose(f, a * lr2 + c, rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(p, 1.0 / (1.0 + np.exp(-(a * lr2 + c))), rtol=1e-15)


def test_unet_concat_order_matters():
    # the same delta placed on the upsampled half's channel 0 sees the (all-zero) deep path
    w = identity_unet_weights()
    w["dec1"][0][0, 16, 2] = 0.0
    w["dec1"][0][0, 0, 2] = 1.0
    h = np.abs(np.random.default_rng(15).normal(0, 3, 4000)) + 1
    f, _ = oracle.unet(w, h)
    np.testing.assert_array_equal(f, np.full(4000, -1.0))


def test_unet_translation_equivariance():
    w = rand_weights(16, 0.0)
    rng = np.random.default_rng(17)
    h = np.zeros(4000)
    h[1500:2500] = np.abs(rng.normal(0, 5, 1000))
    f0, _ = oracle.unet(w, h)
    for shift in (8, 64, 256):
        hs = np.roll(h, shift)
        fs, _ = oracle.unet(w, hs)
        # away from the ends (receptive field is well under 128 bins)
        np.testing.assert_allclose(fs[128 + shift:4000 - 128], f0[128:4000 - 128 - shift],
                                   rtol=1e-12, atol=1e-9)
    # a shift that is not a multiple of 8 breaks the pooling grid: not equivariant
    fs, _ = oracle.unet(w, np.roll(h, 3))
    assert np.max(np.abs(fs[131:3872] - f0[128:3869])) > 1e-6


# ----------------------------------------------------------------- peaks

def _golden_cases():
    with open(os.path.join(GOLDEN, "peaks_handbuilt.json")) as fh:
        return json.load(fh)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_peaks_handbuilt(case):
    f = np.full(4000, case["background"], dtype=np.float64)
    for i, v in case["set"]:
        f[i] = v
    n, z, bins = oracle.peaks(f)
    assert n == len(case["bins"])
    assert list(bins) == case["bins"]
    for zi, want in zip(z, case["z"]):
        if want is not None:
            assert abs(zi - want) < 1e-12
    with np.errstate(over="ignore"):
        rb, rz = ref.peaks(f, 1.0 / (1.0 + np.exp(-f)))
    assert list(rb) == case["bins"]
    np.testing.assert_allclose(z, rz, rtol=0, atol=1e-12)


def test_peaks_truncation_reports_true_count():
    f = np.full(4000, -30.0)
    f[10::20] = 3.0                        # 200 isolated peaks
    n, z, bins = oracle.peaks(f, max_pv=64)
    assert n == 200 and len(z) == 64
    assert list(bins) == list(range(10, 10 + 20 * 64, 20))
    assert np.all(np.diff(z) > 0)


def test_peaks_threshold_equivalence_on_probability():
    # the logit rule p > 0.01 <=> f > ln(0.01/0.99), checked away from the boundary
    rng = np.random.default_rng(18)
    f = rng.normal(-4.6, 2.0, 4000)
    n, _, bins = oracle.peaks(f)
    p = 1.0 / (1.0 + np.exp(-f))
    for i in bins:
        assert p[i] > 0.01
    rb, _ = ref.peaks(f, p)
    assert list(rb) == list(bins)


# ----------------------------------------------------------------- whole pipeline

def test_infer_matches_torch_statement_two_events():
    w = rand_weights(20, 0.05)
    ev = synth.generate_standard(2, 21)
    r = oracle.infer(w, ev.features, ev.offsets, max_pv=1024, want_hist=True,
                     want_logit=True, want_prob=True)
    for e in range(2):
        feats = ev.features[:, ev.offsets[e]:ev.offsets[e + 1]]
        h = ref.histogram(w, feats)
        np.testing.assert_allclose(r["hist"][e], h, rtol=1e-12, atol=1e-12)
        f, p = ref.unet(w, h)
        scale = np.max(np.abs(f))
        np.testing.assert_allclose(r["logit"][e], f, rtol=0, atol=1e-11 * scale)
        bins, z = ref.peaks(f, p)
        n = r["pv_count"][e]
        # decisions can only differ where two logits tie to within rounding
        assert abs(n - len(bins)) <= 1
        if n == len(bins):
            np.testing.assert_allclose(r["pv_z"][e, :n], z, rtol=0, atol=1e-9)


def test_infer_bypasses_invalid_events_and_threads_agree():
    w = rand_weights(22, 0.0)
    ev = synth.generate_standard(6, 23)
    off = ev.offsets.copy()
    off[3] = off[2] - 1                      # event 2 has a negative track count
    r1 = oracle.infer(w, ev.features, off, max_pv=1024, nthreads=1, want_hist=True)
    r4 = oracle.infer(w, ev.features, off, max_pv=1024, nthreads=4, want_hist=True)
    assert r1["pv_count"][2] == -1
    np.testing.assert_array_equal(r1["pv_count"], r4["pv_count"])
    np.testing.assert_array_equal(r1["hist"], r4["hist"])
    ok = [e for e in range(6) if e != 2]
    np.testing.assert_array_equal(np.nan_to_num(r1["pv_z"][ok]), np.nan_to_num(r4["pv_z"][ok]))
    # per-event track cap
    r = oracle.infer(w, ev.features, ev.offsets, max_pv=8, max_tracks_per_event=100)
    big = ev.tracks_per_event() > 100
    assert np.all(r["pv_count"][big] == -1) and np.all(r["pv_count"][~big] >= 0)


def test_fp16_rounding_emulation_against_binary16():
    """The FP16 form's quantisation emulation (a wiring check for the f16 kernels) against
    values IEEE 754 binary16 fixes: 10 stored mantissa bits with ties to even, saturation
    at the largest finite value 65504 (as the form's stores), NaN kept, subnormals down to
    2^-24."""
    x = torch.tensor([1 + 2 ** -11, 1 + 3 * 2 ** -11, 1 + 2 ** -10, 65504.0, 65519.0, 1e6, -1e6,
                      2 ** -24, 2 ** -26, 3 * 2 ** -25, 0.1], dtype=torch.float64)
    want = [1.0, 1 + 2 ** -9, 1 + 2 ** -10, 65504.0, 65504.0, 65504.0, -65504.0,
            2 ** -24, 0.0, 2 * 2 ** -24, 1638 * 2 ** -14]
    got = ref.q_fp16(x).tolist()
    assert got == want
    assert math.isnan(ref.q_fp16(torch.tensor([float("nan")], dtype=torch.float64)).item())


# ----------------------------------------------------------------- per-interval layout (§3)
# Each interval runs the UNet as its own 104-bin sequence (its 100 bins, two zero bins on
# each side); its 100 central logits fill the interval's bins of the event.

def test_per_interval_identity_closed_form():
    """The identity network is pointwise, so every layout must give its closed form; a
    window offset off by one bin would shift the values."""
    a, c = 0.5, -1.0
    w = identity_unet_weights(a, c)
    h = np.random.default_rng(21).normal(0, 3, 4000)
    f, p = oracle.unet_intervals(w, h)
    lr = np.where(h > 0, h, 0.01 * h)
    lr2 = np.where(lr > 0, lr, 0.01 * lr)
    np.testing.assert_allclose(f, a * lr2 + c, rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(p, 1.0 / (1.0 + np.exp(-f)), rtol=1e-15)


def test_per_interval_matches_torch_statement_on_each_window():
    w = rand_weights(22, 0.2)
    h = np.abs(np.random.default_rng(23).normal(0, 5, 4000))
    f, _ = oracle.unet_intervals(w, h)
    for s in (0, 7, 39):
        win = np.concatenate([np.zeros(2), h[100 * s:100 * s + 100], np.zeros(2)])
        fw, _ = ref.unet(w, win)
        np.testing.assert_allclose(f[100 * s:100 * s + 100], fw[2:102], rtol=1e-11, atol=1e-10)


def test_per_interval_intervals_are_independent():
    w = rand_weights(24, 0.2)
    rng = np.random.default_rng(25)
    h = np.abs(rng.normal(0, 5, 4000))
    f0, _ = oracle.unet_intervals(w, h)
    h2 = h.copy()
    h2[1200:1300] = np.abs(rng.normal(0, 5, 100))        # interval 12 only
    f1, _ = oracle.unet_intervals(w, h2)
    changed = np.nonzero(f0 != f1)[0]
    assert changed.size > 0 and changed.min() >= 1200 and changed.max() < 1300
    # the whole-sequence network, by contrast, sees across the interval edges
    g0, _ = oracle.unet(w, h)
    g1, _ = oracle.unet(w, h2)
    changed = np.nonzero(g0 != g1)[0]
    assert changed.min() < 1200 and changed.max() >= 1300


def test_per_interval_infer_uses_the_assembled_logits():
    w = rand_weights(26, 0.1)
    ev = synth.generate_standard(3, 27)
    r = oracle.infer(w, ev.features, ev.offsets, max_pv=672, want_hist=True, want_logit=True,
                     per_interval=True)
    for e in range(3):
        f, _ = oracle.unet_intervals(w, r["hist"][e])
        np.testing.assert_array_equal(r["logit"][e], f)
        n, z, _ = oracle.peaks(f, max_pv=672)    # weights via numpy's exp: z to the last ulp
        assert r["pv_count"][e] == n
        np.testing.assert_allclose(r["pv_z"][e, :n], z, rtol=0, atol=1e-12)


# ----------------------------------------------------------------- all four steps at once

def test_end_to_end_closed_form():
    """FC weights zero: each track adds softplus(b6[j]) to bin j of its slice. Identity
    UNet: logit = a * hist + c (hist >= 0). b6 peaks at j = 50 and is symmetric about it,
    so each populated slice s gives exactly one vertex, at bin 100 s + 50 with a zero
    centroid offset; empty bins stay below the threshold (sigmoid(-6) < 0.01)."""
    a, c = 0.5, -6.0
    w = identity_unet_weights(a, c)
    j = np.arange(100)
    b6 = (3.0 - (j - 50.0) ** 2 / 20.0).astype(np.float32)
    w["fc6"] = (w["fc6"][0], b6)
    counts = {3: 1, 7: 2, 20: 5, 39: 3}
    z = [np.float32(-100 + 10 * s + 4.2) for s, n in counts.items() for _ in range(n)]
    f = np.random.default_rng(30).normal(0, 1, (9, len(z))).astype(np.float32)
    f[2] = z
    r = oracle.infer(w, f, np.array([0, len(z)], np.int32), max_pv=64, want_hist=True,
                     want_logit=True)
    sp = np.logaddexp(0.0, b6.astype(np.float64))
    want_hist = np.zeros(4000)
    for s, n in counts.items():
        want_hist[100 * s:100 * s + 100] = n * sp
    np.testing.assert_allclose(r["hist"][0], want_hist, rtol=1e-14, atol=0)
    np.testing.assert_allclose(r["logit"][0], a * want_hist + c, rtol=1e-14, atol=1e-14)
    assert r["pv_count"][0] == len(counts)
    want_z = [-100.0 + (100 * s + 50 + 0.5) * 0.1 for s in sorted(counts)]
    np.testing.assert_allclose(r["pv_z"][0, :len(counts)], want_z, rtol=0, atol=1e-12)

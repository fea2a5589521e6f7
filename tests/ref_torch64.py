"""A second, independently written float64 statement of PVFinder inference, test-only.

Built from PyTorch CPU library routines (F.linear, F.conv1d, F.conv_transpose1d,
F.max_pool1d, F.softplus, torch.sigmoid) in float64 rather than the oracle's direct
loops, so that a wiring mistake in one (a transposed weight, a wrong concat order, an
off-by-one padding) shows up as a disagreement between the two. It follows §2 of the
paper with the same readings as the oracle. Used only to pin the oracle.
"""

from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

NBINS = 4000


def _t(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float64))


def slice_of(z32: np.ndarray) -> np.ndarray:
    """Slice index from float32 z, float32 round-to-nearest arithmetic; -1 outside."""
    z32 = np.asarray(z32, dtype=np.float32)
    with np.errstate(invalid="ignore"):
        q = (z32 + np.float32(100.0)) / np.float32(10.0)
        ok = np.isfinite(q) & (q >= 0) & (q < 40)
    s = np.full(z32.shape, -1, dtype=np.int64)
    s[ok] = np.floor(q[ok]).astype(np.int64)
    return s


def fc_net(w: dict, x: torch.Tensor) -> torch.Tensor:
    """x [n, 9] float64 -> [n, 100]."""
    h = x
    for i in range(1, 6):
        W, b = w[f"fc{i}"]
        h = F.leaky_relu(F.linear(h, _t(W), _t(b)), 0.01)
    W, b = w["fc6"]
    return F.softplus(F.linear(h, _t(W), _t(b)), beta=1.0, threshold=20.0)


def histogram(w: dict, feats: np.ndarray) -> np.ndarray:
    """One event's [4000] histogram from float32 features [9, n]."""
    feats = np.asarray(feats, dtype=np.float32)
    s = slice_of(feats[2])
    ok = (s >= 0) & np.all(np.isfinite(feats), axis=0)
    x = feats[:, ok].astype(np.float64).T.copy()
    s = s[ok]
    x[:, 2] = x[:, 2] - (-100.0 + 10.0 * s)
    out = fc_net(w, _t(x)).numpy() if x.shape[0] else np.zeros((0, 100))
    hist = np.zeros((40, 100), dtype=np.float64)
    np.add.at(hist, s, out)
    return hist.reshape(-1)


def unet(w: dict, hist: np.ndarray):
    """(logit [L], prob [L]) for one event."""
    def conv(x, name):
        W, b = w[name]
        return F.conv1d(x, _t(W), _t(b), padding=2)

    def up(x, name):
        W, b = w[name]
        return F.leaky_relu(F.conv_transpose1d(x, _t(W), _t(b), stride=2), 0.01)

    lr = lambda v: F.leaky_relu(v, 0.01)
    x = _t(hist).reshape(1, 1, -1)
    e1 = lr(conv(x, "enc1"))
    e2 = lr(conv(F.max_pool1d(e1, 2), "enc2"))
    e3 = lr(conv(F.max_pool1d(e2, 2), "enc3"))
    e4 = lr(conv(F.max_pool1d(e3, 2), "enc4"))
    d3 = lr(conv(torch.cat([up(e4, "up3"), e3], dim=1), "dec3"))
    d2 = lr(conv(torch.cat([up(d3, "up2"), e2], dim=1), "dec2"))
    d1 = lr(conv(torch.cat([up(d2, "up1"), e1], dim=1), "dec1"))
    f = conv(d1, "final").reshape(-1)
    return f.numpy(), torch.sigmoid(f).numpy()


def peaks(f: np.ndarray, p: np.ndarray, thr: float = 0.01):
    """Vectorised local-max rule on the logits; returns (bins, z)."""
    L = f.shape[0]
    tl = np.log(thr / (1.0 - thr))
    big = np.full(5, -np.inf)
    fp = np.concatenate([big, f, big])
    cand = f > tl
    for d in range(1, 6):
        cand &= f > fp[5 - d:5 - d + L]          # left neighbours strictly lower
        cand &= f >= fp[5 + d:5 + d + L]         # right neighbours not higher
    bins = np.nonzero(cand)[0]
    zc = -100.0 + (np.arange(L) + 0.5) * 0.1
    z = []
    for i in bins:
        lo, hi = max(0, i - 3), min(L, i + 4)
        z.append(np.dot(p[lo:hi], zc[lo:hi]) / p[lo:hi].sum())
    return bins, np.array(z)


def unet_quantized(w: dict, hist: np.ndarray, q):
    """The UNet in float64 with q() applied wherever the tensor-core forms store a
    reduced-precision tensor: every GEMM operand (activations and weights) including the
    fused ConvT operands (e4, d3, d2). enc1 and the final conv keep float32 weights, and
    the final conv reads d1 unrounded (it runs in dec1's epilogue). Used to check the
    kernels' wiring tightly, not as the oracle."""
    def conv(x, name, quant_w=True):
        W, b = w[name]
        Wt = _t(W)
        return F.conv1d(x, q(Wt) if quant_w else Wt, _t(b), padding=2)

    def up(x, name):
        W, b = w[name]
        return F.leaky_relu(F.conv_transpose1d(x, q(_t(W)), _t(b), stride=2), 0.01)

    lr = lambda v: F.leaky_relu(v, 0.01)
    x = _t(hist).reshape(1, 1, -1)
    e1 = q(lr(conv(x, "enc1", quant_w=False)))
    e2 = q(lr(conv(F.max_pool1d(e1, 2), "enc2")))
    e3 = q(lr(conv(F.max_pool1d(e2, 2), "enc3")))
    e4 = q(lr(conv(F.max_pool1d(e3, 2), "enc4")))
    u3 = q(up(e4, "up3"))
    d3 = q(lr(conv(torch.cat([u3, e3], dim=1), "dec3")))
    u2 = q(up(d3, "up2"))
    d2 = q(lr(conv(torch.cat([u2, e2], dim=1), "dec2")))
    u1 = q(up(d2, "up1"))
    d1 = lr(conv(torch.cat([u1, e1], dim=1), "dec1"))
    f = conv(d1, "final", quant_w=False).reshape(-1)
    return f.numpy()


def q_bf16(t):
    return t.to(torch.bfloat16).to(torch.float64)


def q_fp16(t):
    """Round to nearest even in IEEE half precision, saturating to +-65504 as the FP16
    form's stores do (NaN stays NaN)."""
    return t.clamp(-65504.0, 65504.0).to(torch.float16).to(torch.float64)


def _e4m3(t):
    """Saturating round-to-nearest-even to float8 e4m3 and back to float64."""
    return t.clamp(-448.0, 448.0).to(torch.float8_e4m3fn).to(torch.float64)


def unet_quantized_fp8(w: dict, hist: np.ndarray, act_scale):
    """The UNet in float64 with the FP8 form's quantisation points: every stored
    activation x becomes e4m3(x / s) * s with the per-tensor scale s of its slot (skip
    concat halves share one), every GEMM weight becomes e4m3(W / s_w[co]) * s_w[co] with
    s_w[co] = max |W[co]| / 448 per output channel. enc1 and the final conv stay float32
    and read unrounded inputs. Used to check the FP8 kernels' wiring, not as the oracle."""
    s = [float(v) for v in act_scale]
    qa = lambda t, k: _e4m3(t / s[k]) * s[k]

    def qw_conv(W):
        W = _t(W)
        sw = W.abs().amax(dim=(1, 2), keepdim=True) / 448.0
        sw = torch.where(sw > 0, sw, torch.ones_like(sw))
        return _e4m3(W / sw) * sw

    def qw_up(W):
        W = _t(W)                                     # [Cin][Cout][2]
        sw = W.abs().amax(dim=(0, 2), keepdim=True) / 448.0
        sw = torch.where(sw > 0, sw, torch.ones_like(sw))
        return _e4m3(W / sw) * sw

    def conv(x, name, q=True):
        W, b = w[name]
        return F.conv1d(x, qw_conv(W) if q else _t(W), _t(b), padding=2)

    def up(x, name):
        W, b = w[name]
        return F.leaky_relu(F.conv_transpose1d(x, qw_up(W), _t(b), stride=2), 0.01)

    lr = lambda v: F.leaky_relu(v, 0.01)
    x = _t(hist).reshape(1, 1, -1)
    e1 = qa(lr(conv(x, "enc1", q=False)), 0)
    e2 = qa(lr(conv(F.max_pool1d(e1, 2), "enc2")), 1)
    e3 = qa(lr(conv(F.max_pool1d(e2, 2), "enc3")), 2)
    e4 = qa(lr(conv(F.max_pool1d(e3, 2), "enc4")), 3)
    u3 = qa(up(e4, "up3"), 2)
    d3 = qa(lr(conv(torch.cat([u3, e3], dim=1), "dec3")), 4)
    u2 = qa(up(d3, "up2"), 1)
    d2 = qa(lr(conv(torch.cat([u2, e2], dim=1), "dec2")), 5)
    u1 = qa(up(d2, "up1"), 0)
    d1 = lr(conv(torch.cat([u1, e1], dim=1), "dec1"))
    f = conv(d1, "final", q=False).reshape(-1)
    return f.numpy()


def histogram_quantized(w: dict, feats: np.ndarray, q):
    """One event's histogram with the tensor-core FC's rounding points: features (with
    the slice-relative z formed in float32) and every FC weight through q(), hidden
    activations through q() after each LeakyReLU, the output layer and softplus in
    float64, summed per bin. Checks the tcgen05 FC wiring, not the oracle."""
    feats = np.asarray(feats, dtype=np.float32)
    s = slice_of(feats[2])
    ok = (s >= 0) & np.all(np.isfinite(feats), axis=0)
    x32 = feats[:, ok].T.copy()
    s = s[ok]
    x32[:, 2] = x32[:, 2] - (np.float32(-100.0) + np.float32(10.0) * s.astype(np.float32))
    h = q(_t(x32.astype(np.float64)))
    for i in range(1, 6):
        W, b = w[f"fc{i}"]
        h = q(F.leaky_relu(F.linear(h, q(_t(W)), _t(b)), 0.01))
    W, b = w["fc6"]
    out = F.softplus(F.linear(h, q(_t(W)), _t(b)), beta=1.0, threshold=20.0).numpy()
    hist = np.zeros((40, 100), dtype=np.float64)
    np.add.at(hist, s, out)
    return hist.reshape(-1)
